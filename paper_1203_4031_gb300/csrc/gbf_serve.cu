// Batched solves and the serving loop (host side; every solve runs the same
// device driver as gbf_dsygv_dev / gbf_zhegv_dev).
//
// Workers: each owns a gbf_context (its workspace) and a CUDA stream, so the
// solves of independent problems overlap on the GPU (the guide's first level
// of parallelism -- independent search intervals / problems -- inside one
// device).  Results do not depend on which worker ran a problem or on what
// ran beside it: every launch configuration is a function of the problem
// alone and no floating-point reduction uses atomics.
//
// gbf_batch_solve: the problems are ordered by estimated cost (Ne n^3,
// largest first) and taken from a shared counter by the workers.
// gbf_server_*:    requests queue in arrival order; a request is admitted
// when a worker is idle and its device footprint fits in what is left of
// the HBM budget (a request that can never fit is failed with info -1);
// latency stamps (queue, run) are returned with the result.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gbf_common.cuh"
#include "gbfeast.h"

namespace gbf {
// implemented in gbf_api.cu
int run_problem(gbf_context *h, cudaStream_t st, const gbf_problem *p, gbf_result *r);
size_t problem_footprint(const gbf_problem *p);
}  // namespace gbf

using namespace gbf;
using clk = std::chrono::steady_clock;

static double ms_since(clk::time_point a, clk::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Worker {
  gbf_context *h = nullptr;
  cudaStream_t st = nullptr;
};

static int make_workers(int count, std::vector<Worker> &ws) {
  int dev = 0;
  cudaGetDevice(&dev);
  for (int i = 0; i < count; ++i) {
    Worker w;
    if (gbf_create(&w.h) != 0) return -1;
    if (cudaStreamCreateWithFlags(&w.st, cudaStreamNonBlocking) != cudaSuccess) return -4;
    ws.push_back(w);
  }
  return 0;
}

static void free_workers(std::vector<Worker> &ws) {
  for (auto &w : ws) {
    if (w.st) cudaStreamSynchronize(w.st), cudaStreamDestroy(w.st);
    if (w.h) gbf_destroy(w.h);
  }
  ws.clear();
}

extern "C" int gbf_batch_solve(gbf_handle h, void *stream, int nprob, const gbf_problem *probs, gbf_result *outs,
                               int nworkers) {
  (void)h;
  if (nprob < 0) return -103;
  if (nprob == 0) return 0;
  if (!probs || !outs) return -104;
  if (nworkers < 1) nworkers = 1;
  nworkers = std::min(nworkers, nprob);
  cudaStream_t caller = (cudaStream_t)stream;
  int dev = 0;
  cudaGetDevice(&dev);
  // inputs are ready when the caller's stream reaches this point
  cudaEvent_t ready;
  GBF_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  GBF_CUDA(cudaEventRecord(ready, caller));
  std::vector<int> order(nprob);
  for (int i = 0; i < nprob; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const double ca = (double)probs[a].fpm[1] * probs[a].n * probs[a].n * probs[a].n;
    const double cb = (double)probs[b].fpm[1] * probs[b].n * probs[b].n * probs[b].n;
    return ca > cb;
  });
  std::vector<Worker> ws;
  if (int rc = make_workers(nworkers, ws)) {
    free_workers(ws);
    cudaEventDestroy(ready);
    return rc;
  }
  std::atomic<int> next{0};
  std::vector<std::thread> th;
  for (int t = 0; t < nworkers; ++t)
    th.emplace_back([&, t]() {
      cudaSetDevice(dev);
      Worker &w = ws[t];
      cudaStreamWaitEvent(w.st, ready, 0);
      for (;;) {
        const int k = next.fetch_add(1);
        if (k >= nprob) break;
        const int i = order[k];
        auto t0 = clk::now();
        run_problem(w.h, w.st, &probs[i], &outs[i]);
        outs[i].run_ms = ms_since(t0, clk::now());
        outs[i].queue_ms = 0.0;
      }
    });
  for (auto &x : th) x.join();
  // the caller's stream waits for every worker stream
  for (auto &w : ws) {
    cudaEvent_t done;
    cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
    cudaEventRecord(done, w.st);
    cudaStreamWaitEvent(caller, done, 0);
    cudaEventDestroy(done);
  }
  free_workers(ws);
  cudaEventDestroy(ready);
  int worst = 0;
  for (int i = 0; i < nprob; ++i)
    if (outs[i].info < 0 && worst == 0) worst = outs[i].info;
  return worst;
}

// ------------------------------------------------------------- server --
struct Request {
  unsigned long long ticket;
  gbf_problem prob;
  gbf_result res;
  size_t bytes;
  clk::time_point t_submit;
  bool done = false;
};

struct gbf_server_s {
  size_t budget = 0, in_use = 0;
  int device = 0;
  std::vector<Worker> workers;
  std::vector<std::thread> threads;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request *> queue;
  std::unordered_map<unsigned long long, Request *> table;
  unsigned long long next_ticket = 1;
  bool stop = false;
  int busy = 0;
  size_t peak = 0;
};

static void server_loop(gbf_server_s *s, int wid) {
  cudaSetDevice(s->device);
  Worker &w = s->workers[wid];
  for (;;) {
    Request *r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      // admission: the oldest request whose footprint fits the budget
      for (;;) {
        if (s->stop && s->queue.empty()) return;
        if (!s->queue.empty()) {
          Request *head = s->queue.front();
          if (head->bytes > s->budget) {  // can never fit
            s->queue.pop_front();
            head->res.info = -1;
            head->done = true;
            s->cv_done.notify_all();
            continue;
          }
          if (s->in_use + head->bytes <= s->budget) {
            r = head;
            s->queue.pop_front();
            s->in_use += r->bytes;
            s->peak = std::max(s->peak, s->in_use);
            ++s->busy;
            break;
          }
        }
        s->cv_work.wait(lk);
      }
    }
    auto t0 = clk::now();
    r->res.queue_ms = ms_since(r->t_submit, t0);
    run_problem(w.h, w.st, &r->prob, &r->res);
    r->res.run_ms = ms_since(t0, clk::now());
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->in_use -= r->bytes;
      --s->busy;
      r->done = true;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

extern "C" int gbf_server_create(size_t hbm_budget_bytes, int nworkers, gbf_server *out) {
  if (!out) return -103;
  if (nworkers < 1) nworkers = 1;
  gbf_server_s *s = new (std::nothrow) gbf_server_s();
  if (!s) return -1;
  s->budget = hbm_budget_bytes;
  cudaGetDevice(&s->device);
  if (int rc = make_workers(nworkers, s->workers)) {
    free_workers(s->workers);
    delete s;
    return rc;
  }
  for (int i = 0; i < nworkers; ++i) s->threads.emplace_back(server_loop, s, i);
  *out = s;
  return 0;
}

extern "C" int gbf_server_submit(gbf_server s, const gbf_problem *p, unsigned long long *ticket) {
  if (!s || !p || !ticket) return -101;
  Request *r = new (std::nothrow) Request();
  if (!r) return -1;
  r->prob = *p;
  r->res = gbf_result{};
  r->bytes = problem_footprint(p);
  r->t_submit = clk::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->ticket = s->next_ticket++;
    s->table[r->ticket] = r;
    s->queue.push_back(r);
  }
  s->cv_work.notify_all();
  *ticket = r->ticket;
  return 0;
}

// 0: done (result copied, ticket released), 1: still queued or running,
// -101: unknown ticket.
extern "C" int gbf_server_poll(gbf_server s, unsigned long long ticket, gbf_result *out) {
  if (!s) return -101;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->table.find(ticket);
  if (it == s->table.end()) return -101;
  if (!it->second->done) return 1;
  if (out) *out = it->second->res;
  delete it->second;
  s->table.erase(it);
  return 0;
}

extern "C" int gbf_server_wait(gbf_server s, unsigned long long ticket, gbf_result *out) {
  if (!s) return -101;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->table.find(ticket);
  if (it == s->table.end()) return -101;
  Request *r = it->second;
  s->cv_done.wait(lk, [&] { return r->done; });
  if (out) *out = r->res;
  delete r;
  s->table.erase(it);
  return 0;
}

extern "C" int gbf_server_stats(gbf_server s, size_t *in_use, size_t *peak, int *queued, int *running) {
  if (!s) return -101;
  std::lock_guard<std::mutex> lk(s->mu);
  if (in_use) *in_use = s->in_use;
  if (peak) *peak = s->peak;
  if (queued) *queued = (int)s->queue.size();
  if (running) *running = s->busy;
  return 0;
}

extern "C" int gbf_server_destroy(gbf_server s) {
  if (!s) return 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto &t : s->threads) t.join();
  free_workers(s->workers);
  for (auto &kv : s->table) delete kv.second;
  delete s;
  return 0;
}
