// rqa_server.cpp -- continuous batching of RQA requests (rqa_server_* of
// include/rqa.h).
//
// Requests are copied at submission and queued in arrival order.  Worker
// threads, each owning an engine with its own CUDA streams and device arena,
// repeatedly admit the longest prefix of the queue whose device memory fits
// in what is left of the budget (and the free slots) and whose work stays
// below an epoch size, run it as one launch epoch (all kernels of all
// admitted series in one submission), and publish the results.  An epoch
// formed from requests that arrived while other epochs run goes to the
// device at once on its worker's streams, so work of different epochs
// overlaps, while four workers keep the number of epochs sharing the GPU low.  Per-request histograms and boundary
// state live in the epoch's device arena until the epoch completes.
#include <chrono>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/rqa.h"
#include "rqa_engine.h"

namespace {

struct Request {
  uint64_t ticket = 0;
  rqa_settings st{};
  std::vector<double> series;
  size_t bytes = 0;
  double cells = 0.0;  // n^2, the epoch-sizing estimate of its GPU work
  int status = RQA_PENDING;
  rqa_measures_t meas{};
  bool queued = true;
};

}  // namespace

struct rqa_server {
  size_t budget = 0;
  int32_t max_slots = 0;
  int workers_n = 4;
  // An epoch stops admitting once it holds this many matrix cells (about 10 ms
  // of tile-kernel work), so epochs stay short and a request that arrives
  // while one runs is picked up by the next free worker.
  double epoch_cells = 1.5e10;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<Request>> all;
  uint64_t next_ticket = 1;
  size_t in_use = 0;
  int32_t slots_used = 0;
  int64_t admitted = 0, completed = 0, epochs = 0;
  bool stop = false;
  int device = 0;
  std::vector<std::thread> threads;

  void worker(int idx);
};

void rqa_server::worker(int idx) {
  (void)idx;
  rqa::Engine eng(device);
  for (;;) {
    std::vector<std::shared_ptr<Request>> epoch;
    double cells = 0.0;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] { return stop || !queue.empty(); });
      if (stop) return;
      // admit in arrival order while memory and slots allow
      while (!queue.empty()) {
        auto& r = queue.front();
        if (slots_used >= max_slots) break;
        if (in_use + r->bytes > budget) break;
        if (!epoch.empty() && cells + r->cells > epoch_cells) break;
        cells += r->cells;
        in_use += r->bytes;
        ++slots_used;
        r->queued = false;
        epoch.push_back(r);
        queue.pop_front();
      }
      if (epoch.empty()) {
        // the head does not fit now: wait for memory or slots to free up
        cv_work.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
      admitted += static_cast<int64_t>(epoch.size());
      ++epochs;
    }
    std::vector<rqa::SeriesInput> in(epoch.size());
    for (size_t q = 0; q < epoch.size(); ++q) {
      in[q].st = epoch[q]->st;
      in[q].host = epoch[q]->series.data();
      in[q].N = static_cast<int64_t>(epoch[q]->series.size());
    }
    std::vector<rqa::SeriesResult> res;
    const int rc = eng.run(in, res, nullptr, rqa::Engine::kNoGraph);
    // the budget bounds the memory of the admitted requests; an engine's
    // arena outlives its epoch, so one larger than the worker's share of the
    // budget is released, and the arenas held between epochs stay within it
    if (eng.arena_bytes() > budget / static_cast<size_t>(workers_n)) eng.release_arena();
    {
      std::lock_guard<std::mutex> lk(mu);
      for (size_t q = 0; q < epoch.size(); ++q) {
        Request& r = *epoch[q];
        r.status = q < res.size() ? res[q].status : (rc != RQA_OK ? rc : RQA_ECUDA);
        if (r.status == RQA_OK) r.meas = res[q].meas;
        std::vector<double>().swap(r.series);
        in_use -= r.bytes;
        --slots_used;
        ++completed;
      }
    }
    cv_done.notify_all();
    cv_work.notify_all();
  }
}

extern "C" {

int rqa_server_create(size_t mem_budget_bytes, int32_t max_slots, rqa_server** out) {
  if (!out || mem_budget_bytes == 0 || max_slots < 1) return RQA_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
    cudaGetLastError();
    return RQA_ENODEV;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3) return RQA_ENODEV;
  // every kernel loaded before the first request: a lazy load in the middle
  // of other requests' work stalls them all
  const int pre = rqa_preload_kernels(nullptr);
  if (pre != RQA_OK) return pre;
  rqa_server* s = new (std::nothrow) rqa_server();
  if (!s) return RQA_ENOMEM;
  s->budget = mem_budget_bytes;
  s->max_slots = max_slots;
  s->device = dev;
  // measured on the served mix (8 s Poisson streams): four workers keep p99
  // at 46 ms at 200 req/s and 129 ms at 400 req/s (sixteen: 57 and 313 ms,
  // their epochs sharing the GPU) and serve the most at 600 req/s (491/s)
  s->workers_n = 4;
  if (const char* e = std::getenv("RQA_SERVE_WORKERS")) {  // tuning override
    const int w = std::atoi(e);
    if (w >= 1 && w <= 32) s->workers_n = w;
  }
  if (const char* e = std::getenv("RQA_SERVE_EPOCH_CELLS")) {
    const double c = std::atof(e);
    if (c > 0) s->epoch_cells = c;
  }
  for (int w = 0; w < s->workers_n; ++w) s->threads.emplace_back(&rqa_server::worker, s, w);
  *out = s;
  return RQA_OK;
}

int rqa_submit(rqa_server* s, const rqa_settings* settings, const double* host_series, int64_t n,
               uint64_t* ticket) {
  if (!s || !host_series || !ticket) return RQA_EINVAL;
  std::string msg;
  int rc = rqa::validate_settings(settings, &msg);
  if (rc != RQA_OK) return rc;
  const int64_t nv = n - static_cast<int64_t>(settings->m - 1) * settings->tau;
  if (n < 1 || nv < 1) return RQA_ESHORT;
  if (nv > RQA_MAX_N) return RQA_ETOOBIG;
  auto r = std::make_shared<Request>();
  r->st = *settings;
  r->bytes = rqa::series_device_bytes(*settings, n);
  r->cells = static_cast<double>(nv) * static_cast<double>(nv);
  if (r->bytes > s->budget) return RQA_ENOMEM;
  r->series.assign(host_series, host_series + n);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->ticket = s->next_ticket++;
    *ticket = r->ticket;
    s->all.emplace(r->ticket, r);
    s->queue.push_back(r);
  }
  s->cv_work.notify_one();
  return RQA_OK;
}

int rqa_poll(rqa_server* s, uint64_t ticket, rqa_measures_t* out) {
  if (!s) return RQA_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return RQA_ENOTFOUND;
  const Request& r = *it->second;
  if (r.status == RQA_OK && out) *out = r.meas;
  return r.status;
}

int rqa_wait(rqa_server* s, uint64_t ticket, int64_t timeout_ms, rqa_measures_t* out) {
  if (!s) return RQA_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return RQA_ENOTFOUND;
  std::shared_ptr<Request> r = it->second;
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
  while (r->status == RQA_PENDING) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) break;
  }
  if (r->status == RQA_OK && out) *out = r->meas;
  return r->status;
}

int rqa_release(rqa_server* s, uint64_t ticket) {
  if (!s) return RQA_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return RQA_ENOTFOUND;
  std::shared_ptr<Request> r = it->second;
  if (r->status == RQA_PENDING) {
    if (!r->queued) return RQA_PENDING;  // running: cannot cancel
    for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
      if ((*q)->ticket == ticket) {
        s->queue.erase(q);
        break;
      }
  }
  s->all.erase(it);
  return RQA_OK;
}

int rqa_server_counters(rqa_server* s, int64_t* admitted, int64_t* completed, int64_t* queued,
                        int64_t* in_flight, int64_t* bytes_in_use, int64_t* epochs) {
  if (!s) return RQA_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (admitted) *admitted = s->admitted;
  if (completed) *completed = s->completed;
  if (queued) *queued = static_cast<int64_t>(s->queue.size());
  if (in_flight) *in_flight = s->slots_used;
  if (bytes_in_use) *bytes_in_use = static_cast<int64_t>(s->in_use);
  if (epochs) *epochs = s->epochs;
  return RQA_OK;
}

void rqa_server_destroy(rqa_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->threads) t.join();
  delete s;
}

}  // extern "C"
