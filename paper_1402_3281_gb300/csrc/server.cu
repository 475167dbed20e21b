// server.cu -- a request loop that serves partition requests by continuous
// batching (no counterpart in the paper, whose partitioner handles one graph
// per run).
//
// Requests are copied in at submit time and queued in arrival order.  Worker
// threads (one CUDA stream each) take the longest run of queued requests from
// the front whose estimated device memory fits in what the budget has left,
// and partition them as one batch (sclap_partition_batch).  With several
// workers, requests that arrive while a batch is on the GPU start in another
// batch as soon as budget is free, and the two batches overlap on the
// device.  Every result equals the one the same request gets alone, because
// a batched graph's arithmetic does not depend on its batch.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>

#include "common.cuh"

namespace sclap {
void record_last_error(const char* msg);   // driver.cu
}

namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { QUEUED, RUNNING, DONE };

struct Request {
  int64_t id = 0, n = 0, m = 0, est = 0;
  int32_t k = 1;
  double eps = 0;
  uint64_t seed = 0;
  std::vector<int64_t> row_ptr;
  std::vector<int32_t> col, node_w, edge_w;   // empty weights: unit
  std::vector<int32_t> block;
  int64_t cut = 0, max_bw = 0;
  int32_t status = SCLAP_OK;
  ReqState state = QUEUED;
  Clock::time_point t_submit, t_done;
};

// Device bytes a request may hold while it runs: its level-0 graph, the
// coarse levels (at most as large again), per-node LP and contraction
// scratch, and the contraction table (8 B per slot, at most 4 slots per arc).
int64_t estimate_bytes(int64_t n, int64_t m) {
  return 320 * n + 64 * m + (1 << 16);
}

}  // namespace

struct sclap_server {
  sclap_config cfg{};
  int64_t budget = 0;
  int32_t max_batch = 0;
  int64_t linger_us = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work;   // workers: queue or budget changed
  std::condition_variable cv_done;   // pollers: a request finished
  std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
  std::deque<Request*> queue;
  int64_t next_id = 0;
  int64_t inflight = 0;              // estimated bytes of running requests
  bool stop = false;
  std::vector<std::thread> workers;

  bool head_fits() const {
    return !queue.empty() && (inflight == 0 || inflight + queue.front()->est <= budget);
  }
  void worker_main();
};

void sclap_server::worker_main() {
  cudaSetDevice(device);
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) st = nullptr;
  std::vector<Request*> batch;
  std::vector<sclap_graph> gs;
  for (;;) {
    batch.clear();
    int64_t taken = 0;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] { return stop || head_fits(); });
      if (stop) break;
      if (linger_us > 0 && (int64_t)queue.size() < max_batch) {
        // let a partial batch fill for a moment before starting it
        cv_work.wait_for(lk, std::chrono::microseconds(linger_us),
                         [&] { return stop || (int64_t)queue.size() >= max_batch; });
        if (stop) break;
        if (!head_fits()) continue;
      }
      while (!queue.empty() && (int64_t)batch.size() < max_batch) {
        Request* r = queue.front();
        if (inflight + taken > 0 && inflight + taken + r->est > budget) break;
        queue.pop_front();
        r->state = RUNNING;
        taken += r->est;
        batch.push_back(r);
      }
      inflight += taken;
    }
    gs.assign(batch.size(), sclap_graph{});
    for (size_t i = 0; i < batch.size(); ++i) {
      Request* r = batch[i];
      r->block.assign((size_t)r->n, 0);
      sclap_graph& g = gs[i];
      g.n = r->n;
      g.row_ptr = r->row_ptr.data();
      g.col = r->col.empty() ? nullptr : r->col.data();
      g.node_w = r->node_w.empty() ? nullptr : r->node_w.data();
      g.edge_w = r->edge_w.empty() ? nullptr : r->edge_w.data();
      g.k = r->k;
      g.eps = r->eps;
      g.seed = r->seed;
      g.block_out = r->block.data();
    }
    const int rc = st ? sclap_partition_batch((int32_t)gs.size(), gs.data(), &cfg, 0, st)
                      : SCLAP_ECUDA;
    {
      std::lock_guard<std::mutex> lk(mu);
      const Clock::time_point now = Clock::now();
      for (size_t i = 0; i < batch.size(); ++i) {
        Request* r = batch[i];
        // a failure of the whole call (not of one graph) is reported to all
        r->status = (rc != SCLAP_OK && gs[i].status == SCLAP_OK) ? rc : gs[i].status;
        r->cut = gs[i].cut;
        r->max_bw = gs[i].max_block_weight;
        r->t_done = now;
        r->state = DONE;
        r->row_ptr = {};
        r->col = {};
        r->node_w = {};
        r->edge_w = {};
      }
      inflight -= taken;
    }
    cv_done.notify_all();
    cv_work.notify_all();
  }
  if (st) cudaStreamDestroy(st);
}

namespace {

template <class F>
int server_guard(F&& f) {
  try {
    f();
    sclap::record_last_error("");
    return SCLAP_OK;
  } catch (const sclap::Error& e) {
    sclap::record_last_error(e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    sclap::record_last_error("host out of memory");
    return SCLAP_ENOMEM;
  } catch (const std::exception& e) {
    sclap::record_last_error(e.what());
    return SCLAP_EINTERNAL;
  }
}

}  // namespace

extern "C" {

int sclap_server_create(const sclap_config* cfg, const sclap_server_options* opts,
                        sclap_server** out) {
  return server_guard([&] {
    using sclap::Error;
    if (!out) throw Error(SCLAP_EINVAL, "NULL out");
    *out = nullptr;
    sclap_server_options o{};
    if (opts) o = *opts;
    if (o.device_budget_bytes < 0 || o.workers < 0 || o.workers > 16 || o.max_batch < 0 ||
        o.linger_us < 0)
      throw Error(SCLAP_EINVAL, "bad server option");
    std::unique_ptr<sclap_server> S(new sclap_server());
    if (cfg) S->cfg = *cfg;
    else sclap_default_config(&S->cfg);
    S->budget = o.device_budget_bytes ? o.device_budget_bytes : ((int64_t)120 << 30);
    S->max_batch = o.max_batch ? o.max_batch : 512;
    S->linger_us = o.linger_us;
    SCLAP_CUDA(cudaGetDevice(&S->device));
    const int nw = o.workers ? o.workers : 2;
    for (int i = 0; i < nw; ++i) S->workers.emplace_back([p = S.get()] { p->worker_main(); });
    *out = S.release();
  });
}

int sclap_server_submit(sclap_server* S, int64_t n, const int64_t* row_ptr, const int32_t* col,
                        const int32_t* node_w, const int32_t* edge_w, int32_t k, double eps,
                        uint64_t seed, int64_t* request_id) {
  return server_guard([&] {
    using sclap::Error;
    if (!S || !request_id) throw Error(SCLAP_EINVAL, "NULL argument");
    if (n < 1 || n >= ((int64_t)1 << 31)) throw Error(SCLAP_EINVAL, "n must be in [1, 2^31)");
    if (!row_ptr) throw Error(SCLAP_EINVAL, "NULL row_ptr");
    if (k < 1 || (int64_t)k > n) throw Error(SCLAP_EINVAL, "k must be in [1, n]");
    if (!(eps >= 0.0) || eps > 1e9) throw Error(SCLAP_EINVAL, "eps must be >= 0");
    const int64_t m = row_ptr[n];
    if (m < 0 || row_ptr[0] != 0) throw Error(SCLAP_ECSR, "bad row_ptr");
    if (m > 0 && !col) throw Error(SCLAP_EINVAL, "NULL col with arcs present");
    std::unique_ptr<Request> r(new Request());
    r->n = n;
    r->m = m;
    r->k = k;
    r->eps = eps;
    r->seed = seed;
    r->est = estimate_bytes(n, m);
    if (r->est > S->budget)
      throw Error(SCLAP_ENOMEM, "request needs more device memory than the server's budget");
    r->row_ptr.assign(row_ptr, row_ptr + n + 1);
    if (m > 0) r->col.assign(col, col + m);
    if (node_w) r->node_w.assign(node_w, node_w + n);
    if (edge_w && m > 0) r->edge_w.assign(edge_w, edge_w + m);
    r->t_submit = Clock::now();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      if (S->stop) throw Error(SCLAP_EINVAL, "server is shutting down");
      r->id = S->next_id++;
      *request_id = r->id;
      S->queue.push_back(r.get());
      S->reqs.emplace(r->id, std::move(r));
    }
    S->cv_work.notify_one();
  });
}

int sclap_server_poll(sclap_server* S, int64_t request_id, int32_t timeout_ms, int32_t* block_out,
                      int64_t* cut_out, int64_t* max_block_weight_out, double* latency_ms_out) {
  int status = SCLAP_OK;
  const int rc = server_guard([&] {
    using sclap::Error;
    if (!S) throw Error(SCLAP_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(request_id);
    if (it == S->reqs.end()) throw Error(SCLAP_EINVAL, "unknown request id");
    Request* r = it->second.get();
    auto done = [&] { return r->state == DONE; };
    if (!done()) {
      if (timeout_ms < 0) S->cv_done.wait(lk, done);
      else if (timeout_ms > 0)
        S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done);
    }
    if (!done()) {
      status = SCLAP_PENDING;
      return;
    }
    status = r->status;
    if (status == SCLAP_OK || status == SCLAP_EINFEASIBLE) {
      if (block_out) std::copy(r->block.begin(), r->block.end(), block_out);
      if (cut_out) *cut_out = r->cut;
      if (max_block_weight_out) *max_block_weight_out = r->max_bw;
    }
    if (latency_ms_out)
      *latency_ms_out =
          std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    S->reqs.erase(it);
  });
  return rc != SCLAP_OK ? rc : status;
}

int sclap_server_destroy(sclap_server* S) {
  if (!S) return SCLAP_EINVAL;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  S->cv_done.notify_all();
  for (std::thread& t : S->workers)
    if (t.joinable()) t.join();
  delete S;
  return SCLAP_OK;
}

}  // extern "C"
