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
//
// Results are not copied: a batch's page-locked result buffers leave the
// worker's context with the results in them (bsort_take_result_buffers) and
// stay held until every result of the batch has been released
// (bsort_result_release, from any thread); they then go back to the worker,
// whose next batch writes into them.
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
#include "bsort_dev.cuh"

namespace {

using Clock = std::chrono::steady_clock;

// Device bytes one document of `len` bytes may occupy while in flight: the
// input, letters and word starts, two key buffers (at most 4 bytes of keys
// per input byte), offsets and the sorted stream, plus fixed scratch.
uint64_t footprint(uint64_t len) { return 16 * len + (64u << 10); }

struct Request {
  uint64_t tag;
  std::vector<uint8_t> bytes;   // the document's copy (bsort_submit)
  const uint8_t* ptr = nullptr;  // or the caller's own bytes (bsort_submit_borrowed)
  size_t len = 0;
  uint64_t foot;
  Clock::time_point submitted;
};

struct Worker;

// A batch's result buffers and how many of its results still hold them.
struct BatchHold {
  bsort_host_out* bufs;
  uint32_t refs;
  Worker* owner;
};

struct Done {
  uint64_t tag;
  bsort_result res;  // pointers into its batch's buffers (none for a failed document)
  BatchHold* hold;   // null when res points nowhere
  uint64_t latency_ns;
};

struct Worker {
  bsort_ctx* ctx = nullptr;
  std::vector<bsort_host_out*> free_bufs;  // released result buffers, for the next batch
};

struct Server {
  std::mutex mu;
  std::condition_variable cv_work, cv_space;
  std::deque<Request> queue;
  std::deque<Done> done;
  std::unordered_map<const void*, BatchHold*> handed;  // polled results not yet released, by counts pointer
  uint64_t budget = 0, in_flight = 0;
  uint32_t max_docs = 0;
  bool stop = false;
  bool want_offsets = true;
  std::vector<Worker*> workers;
  std::vector<std::thread> threads;
};

std::mutex g_servers_mu;
std::unordered_map<const bsort_ctx*, Server*> g_servers;

Server* server_of(const bsort_ctx* c) {
  std::lock_guard<std::mutex> lk(g_servers_mu);
  auto it = g_servers.find(c);
  return it == g_servers.end() ? nullptr : it->second;
}

// Ends one result's hold on its batch's buffers (under s->mu); the last one
// gives them back to the worker that filled them, or frees them once the
// workers are gone.
void unhold(Server* s, BatchHold* h) {
  if (--h->refs == 0) {
    if (s->stop)
      bsort_free_result_buffers(h->bufs);
    else
      h->owner->free_bufs.push_back(h->bufs);
    delete h;
  }
}

// Frees every result not yet released, polled or not (the server is stopped).
void free_results(Server* s) {
  std::vector<BatchHold*> holds;
  for (Done& d : s->done)
    if (d.hold) holds.push_back(d.hold);
  for (auto& kv : s->handed) holds.push_back(kv.second);
  std::sort(holds.begin(), holds.end());
  holds.erase(std::unique(holds.begin(), holds.end()), holds.end());
  for (BatchHold* h : holds) {
    bsort_free_result_buffers(h->bufs);
    delete h;
  }
  s->done.clear();
  s->handed.clear();
}

void worker_loop(Server* s, Worker* wk) {
  bsort_ctx* ctx = wk->ctx;
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
      ptrs[i] = batch[i].ptr ? batch[i].ptr : batch[i].bytes.data();
      lens[i] = batch[i].ptr ? batch[i].len : batch[i].bytes.size();
    }
    {
      // result buffers to write into: a set released since an earlier batch
      // that is large enough for this one, else new ones (sized for the
      // whole batch before the call, so that the call grows none of them).
      // A set is never regrown or freed while serving: freeing page-locked
      // memory waits for the whole device, which would stall every worker.
      uint64_t bytes = 0;
      for (size_t i = 0; i < batch.size(); ++i) bytes += lens[i];
      bsort_host_out* reuse = nullptr;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        for (size_t i = wk->free_bufs.size(); i-- > 0;)
          if (bsort_result_buffers_fit(wk->free_bufs[i], bytes, batch.size())) {
            reuse = wk->free_bufs[i];
            wk->free_bufs.erase(wk->free_bufs.begin() + (long)i);
            break;
          }
      }
      if (reuse) bsort_give_result_buffers(ctx, reuse);
      bsort_reserve_result_buffers(ctx, bytes, batch.size());  // (a failure surfaces in the call)
    }
    const bsort_status st = bsort_batch(ctx, ptrs.data(), lens.data(), batch.size(), outs.data());
    BatchHold* hold = new BatchHold{bsort_take_result_buffers(ctx), 0, wk};
    std::vector<Done> finished(batch.size());
    const Clock::time_point now = Clock::now();
    for (size_t i = 0; i < batch.size(); ++i) {
      Done& d = finished[i];
      d.tag = batch[i].tag;
      d.hold = nullptr;
      if (st != BSORT_OK && outs[i].status == BSORT_OK && outs[i].counts == nullptr) {
        // the whole call failed (not one document): report the call's status
        // (every document that succeeded, empty ones included, has counts)
        std::memset(&d.res, 0, sizeof(d.res));
        d.res.status = st;
      } else {
        d.res = outs[i];
        if (d.res.status != BSORT_OK || !d.res.counts) {
          d.res.counts = nullptr;
          d.res.offsets = nullptr;
          d.res.stream = nullptr;
        } else {
          d.hold = hold;
          ++hold->refs;
        }
      }
      d.latency_ns = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(now - batch[i].submitted).count();
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->in_flight -= foot;
      if (hold->refs == 0) {  // no result points into the buffers
        wk->free_bufs.push_back(hold->bufs);
        delete hold;
      }
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
  // the finished results stay (their buffers are their own) until released
  // or until the server is dropped
  std::lock_guard<std::mutex> lk(s->mu);
  for (Worker* w : s->workers) {
    for (bsort_host_out* b : w->free_bufs) bsort_free_result_buffers(b);
    bsort_destroy(w->ctx);
    delete w;
  }
  s->workers.clear();
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
  {
    std::lock_guard<std::mutex> lk(s->mu);
    free_results(s);
  }
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
      for (Worker* x : s->workers) {
        bsort_destroy(x->ctx);
        delete x;
      }
      delete s;
      return st;
    }
    Worker* x = new Worker();
    x->ctx = w;
    s->workers.push_back(x);
  }
  for (Worker* w : s->workers) s->threads.emplace_back(worker_loop, s, w);
  std::lock_guard<std::mutex> lk(g_servers_mu);
  g_servers[ctx] = s;
  return BSORT_OK;
}

static bsort_status submit_request(bsort_ctx* ctx, const uint8_t* bytes, size_t len, uint64_t tag, bool borrow) {
  Server* s = server_of(ctx);
  if (!s || (!bytes && len)) return BSORT_E_INVAL;
  if ((uint64_t)len >= (1ull << 30)) return BSORT_E_TOO_LARGE;
  Request r;
  r.tag = tag;
  if (borrow) {
    r.ptr = len ? bytes : nullptr;
    r.len = len;
  } else {
    r.bytes.assign(bytes, bytes + len);
  }
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

bsort_status bsort_submit(bsort_ctx* ctx, const uint8_t* bytes, size_t len, uint64_t tag) {
  return submit_request(ctx, bytes, len, tag, false);
}

bsort_status bsort_submit_borrowed(bsort_ctx* ctx, const uint8_t* bytes, size_t len, uint64_t tag) {
  return submit_request(ctx, bytes, len, tag, true);
}

size_t bsort_poll(bsort_ctx* ctx, uint64_t* tags, bsort_result* outs, uint64_t* latency_ns, size_t max) {
  Server* s = server_of(ctx);
  if (!s || !tags || !outs) return 0;
  std::lock_guard<std::mutex> lk(s->mu);
  size_t k = 0;
  while (k < max && !s->done.empty()) {
    Done& d = s->done.front();
    tags[k] = d.tag;
    outs[k] = d.res;
    if (latency_ns) latency_ns[k] = d.latency_ns;
    if (d.hold) s->handed[d.res.counts] = d.hold;  // held until bsort_result_release
    s->done.pop_front();
    ++k;
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

bool bsort_serve_release(const bsort_ctx* ctx, const bsort_result* res) {
  if (!res || !res->counts) return false;
  Server* s = server_of(ctx);
  if (!s) return false;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->handed.find(res->counts);
  if (it == s->handed.end()) return false;
  BatchHold* h = it->second;
  s->handed.erase(it);
  unhold(s, h);
  return true;
}
