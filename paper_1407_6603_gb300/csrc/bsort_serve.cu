// Serving: a request loop with continuous batching over the batch path.
//
// bsort_serve_start() starts worker threads; each owns a context of its own
// (its own CUDA stream and device arena).  bsort_submit() copies a document
// into the request queue.  A worker takes the queued requests in arrival
// order, as many as fit its batch size and the device-memory budget of the
// requests in flight, sorts them with one bsort_batch call, and posts each
// result to the completion queue that bsort_poll() drains.  While one
// worker's batch runs on the GPU the next requests gather for the other, so
// requests that arrive during a batch are admitted as soon as a worker and
// enough of the budget are free, and the workers' batches overlap on the
// device.  Every result is the one bsort_text gives for the document alone.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bsort.h"

namespace {

using Clock = std::chrono::steady_clock;

// Device bytes one document of `len` bytes may occupy while in flight: the
// input, letters and word starts, two key buffers (at most 4 bytes of keys
// per input byte), offsets and the sorted stream, plus fixed scratch.
uint64_t footprint(uint64_t len) { return 16 * len + (64u << 10); }

struct Request {
  uint64_t tag;
  std::vector<uint8_t> bytes;
  uint64_t foot;
  Clock::time_point submitted;
};

struct Done {
  uint64_t tag;
  bsort_result res;  // pointers into the vectors below
  std::vector<uint64_t> counts;
  std::vector<uint32_t> offsets;
  std::vector<uint8_t> stream;
  uint64_t latency_ns;
};

struct Server {
  std::mutex mu;
  std::condition_variable cv_work, cv_space;
  std::deque<Request> queue;
  std::deque<Done> done;
  std::vector<Done> polled;  // results handed out by the last poll, kept until the next one
  uint64_t budget = 0, in_flight = 0;
  uint32_t max_docs = 0;
  bool stop = false;
  bool want_offsets = true;
  std::vector<bsort_ctx*> ctxs;
  std::vector<std::thread> threads;
};

std::mutex g_servers_mu;
std::unordered_map<const bsort_ctx*, Server*> g_servers;

Server* server_of(const bsort_ctx* c) {
  std::lock_guard<std::mutex> lk(g_servers_mu);
  auto it = g_servers.find(c);
  return it == g_servers.end() ? nullptr : it->second;
}

void copy_result(const bsort_result& r, Done& d, bool want_offsets) {
  d.res = r;
  if (r.status != BSORT_OK || !r.counts) {
    d.res.counts = nullptr;
    d.res.offsets = nullptr;
    d.res.stream = nullptr;
    return;
  }
  d.counts.assign(r.counts, r.counts + r.max_len + 1);
  if (want_offsets && r.offsets) d.offsets.assign(r.offsets, r.offsets + r.n_words + 1);
  d.stream.assign(r.stream, r.stream + r.stream_bytes);
  d.res.counts = d.counts.data();
  d.res.offsets = d.offsets.empty() ? nullptr : d.offsets.data();
  d.res.stream = d.stream.data();
}

void worker_loop(Server* s, bsort_ctx* ctx) {
  std::vector<Request> batch;
  std::vector<const uint8_t*> ptrs;
  std::vector<size_t> lens;
  std::vector<bsort_result> outs;
  for (;;) {
    batch.clear();
    uint64_t foot = 0;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
      if (s->queue.empty()) return;  // stopping, nothing left
      // admit the oldest requests while they fit the batch and the budget
      while (!s->queue.empty() && batch.size() < s->max_docs) {
        const uint64_t f = s->queue.front().foot;
        if (s->in_flight + f > s->budget) {
          if (!batch.empty()) break;
          // Wait for budget.  Another worker may take the front request
          // meanwhile, so the loop looks at the queue afresh after the wait.
          s->cv_space.wait(lk, [&] {
            return s->stop || s->queue.empty() || s->in_flight + s->queue.front().foot <= s->budget;
          });
          if (s->stop && (s->queue.empty() || s->in_flight + s->queue.front().foot > s->budget)) return;
          continue;
        }
        s->in_flight += f;
        foot += f;
        batch.push_back(std::move(s->queue.front()));
        s->queue.pop_front();
      }
    }
    if (batch.empty()) continue;  // the queue emptied while this worker waited
    ptrs.resize(batch.size());
    lens.resize(batch.size());
    outs.assign(batch.size(), bsort_result{});
    for (size_t i = 0; i < batch.size(); ++i) {
      ptrs[i] = batch[i].bytes.data();
      lens[i] = batch[i].bytes.size();
    }
    const bsort_status st = bsort_batch(ctx, ptrs.data(), lens.data(), batch.size(), outs.data());
    std::vector<Done> finished(batch.size());
    const Clock::time_point now = Clock::now();
    for (size_t i = 0; i < batch.size(); ++i) {
      Done& d = finished[i];
      d.tag = batch[i].tag;
      if (st != BSORT_OK && outs[i].status == BSORT_OK && outs[i].counts == nullptr) {
        // the whole call failed (not one document): report the call's status
        // (every document that succeeded, empty ones included, has counts)
        std::memset(&d.res, 0, sizeof(d.res));
        d.res.status = st;
      } else {
        copy_result(outs[i], d, s->want_offsets);
      }
      d.latency_ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(now - batch[i].submitted).count();
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->in_flight -= foot;
      for (Done& d : finished) s->done.push_back(std::move(d));
    }
    s->cv_space.notify_all();
  }
}

void stop_server(Server* s) {
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  s->cv_space.notify_all();
  for (std::thread& t : s->threads) t.join();
  s->threads.clear();
  for (bsort_ctx* c : s->ctxs) bsort_destroy(c);
  s->ctxs.clear();
}

}  // namespace

// Called by bsort_destroy: stops the context's server, if any.
void bsort_serve_shutdown(const bsort_ctx* ctx) {
  Server* s = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_servers_mu);
    auto it = g_servers.find(ctx);
    if (it == g_servers.end()) return;
    s = it->second;
    g_servers.erase(it);
  }
  stop_server(s);
  delete s;
}

extern "C" {

void bsort_serve_config_default(bsort_serve_config* cfg) {
  if (!cfg) return;
  cfg->hbm_budget = 64ull << 30;
  cfg->workers = 2;
  cfg->max_batch_docs = 1024;
}

bsort_status bsort_serve_start(bsort_ctx* ctx, const bsort_serve_config* cfg) {
  if (!ctx) return BSORT_E_INVAL;
  bsort_serve_config conf;
  bsort_serve_config_default(&conf);
  if (cfg) conf = *cfg;
  if (conf.hbm_budget == 0) conf.hbm_budget = 64ull << 30;
  if (conf.workers == 0) conf.workers = 2;
  if (conf.max_batch_docs == 0) conf.max_batch_docs = 1024;
  if (conf.workers > 16) return BSORT_E_INVAL;
  if (Server* old = server_of(ctx)) {
    {
      std::lock_guard<std::mutex> lk(old->mu);
      if (!old->stop) return BSORT_E_BUSY;  // already serving
    }
    bsort_serve_shutdown(ctx);  // a stopped server: drop it and its unpolled results
  }
  bsort_config wc;
  bsort_config_default(&wc);
  if (bsort_context_config(ctx, &wc) != BSORT_OK) return BSORT_E_INVAL;
  wc.profile = 0;
  Server* s = new Server();
  s->budget = conf.hbm_budget;
  s->max_docs = conf.max_batch_docs;
  s->want_offsets = wc.want_offsets != 0;
  for (uint32_t i = 0; i < conf.workers; ++i) {
    bsort_ctx* w = nullptr;
    const bsort_status st = bsort_create(&w, &wc);
    if (st != BSORT_OK) {
      for (bsort_ctx* c : s->ctxs) bsort_destroy(c);
      delete s;
      return st;
    }
    s->ctxs.push_back(w);
  }
  for (bsort_ctx* w : s->ctxs) s->threads.emplace_back(worker_loop, s, w);
  std::lock_guard<std::mutex> lk(g_servers_mu);
  g_servers[ctx] = s;
  return BSORT_OK;
}

bsort_status bsort_submit(bsort_ctx* ctx, const uint8_t* bytes, size_t len, uint64_t tag) {
  Server* s = server_of(ctx);
  if (!s || (!bytes && len)) return BSORT_E_INVAL;
  if ((uint64_t)len >= (1ull << 30)) return BSORT_E_TOO_LARGE;
  Request r;
  r.tag = tag;
  r.bytes.assign(bytes, bytes + len);
  r.foot = footprint(len);
  if (r.foot > s->budget) return BSORT_E_TOO_LARGE;
  r.submitted = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return BSORT_E_BUSY;
    s->queue.push_back(std::move(r));
  }
  s->cv_work.notify_one();
  return BSORT_OK;
}

size_t bsort_poll(bsort_ctx* ctx, uint64_t* tags, bsort_result* outs, uint64_t* latency_ns, size_t max) {
  Server* s = server_of(ctx);
  if (!s || !tags || !outs) return 0;
  std::lock_guard<std::mutex> lk(s->mu);
  s->polled.clear();  // results of the previous poll are released here
  size_t k = 0;
  while (k < max && !s->done.empty()) {
    s->polled.push_back(std::move(s->done.front()));
    s->done.pop_front();
    ++k;
  }
  for (size_t i = 0; i < k; ++i) {
    Done& d = s->polled[i];
    tags[i] = d.tag;
    outs[i] = d.res;
    if (latency_ns) latency_ns[i] = d.latency_ns;
  }
  return k;
}

size_t bsort_serve_pending(const bsort_ctx* ctx) {
  Server* s = server_of(ctx);
  if (!s) return 0;
  std::lock_guard<std::mutex> lk(s->mu);
  return s->queue.size();
}

bsort_status bsort_serve_stop(bsort_ctx* ctx) {
  Server* s = server_of(ctx);
  if (!s) return BSORT_E_INVAL;
  // finish the queued requests, then stop the workers; unpolled results stay
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_space.notify_all();
  }
  for (;;) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->queue.empty() && s->in_flight == 0) break;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
  stop_server(s);
  return BSORT_OK;
}

}  // extern "C"
