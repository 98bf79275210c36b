// Serving loop: continuous batching of cooling runs (contract in include/peps_vmc.h).
//
// A scheduler admits queued requests in arrival order under a device-memory budget and a
// cap on running requests; each admitted request runs on its own context, stream and host
// worker thread, so concurrent requests overlap on the GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/peps_vmc.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int id = 0;
  peps_request req{};
  size_t footprint = 0;
  int state = PEPS_REQ_QUEUED;
  std::vector<peps_stats> steps;
  std::vector<double> step_ms;
  std::vector<double> theta;
  std::thread worker;
};

}  // namespace

struct peps_server {
  size_t budget = 0, used = 0;
  int max_active = 1, active = 0, blocks = 0, device = 0;
  int next_id = 1;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<int> queue;
  std::map<int, std::unique_ptr<Request>> reqs;
  std::vector<double> all_ms;
  long long samples = 0;
  bool started = false;
  bool stopping = false;   // peps_srv_stop: cancel the queue, end running requests after a step
  Clock::time_point t_first, t_last;
};

namespace {

void admit(peps_server* s);

// Runs one request to its end time (worker thread).
void run_request(peps_server* s, Request* r) {
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  int state = PEPS_REQ_DONE;
  peps_ctx* ctx = nullptr;
  peps_params P = r->req.params;
  if (s->blocks > 0 && P.n_blocks == 0) P.n_blocks = s->blocks;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      peps_init(&P, st, &ctx) != PEPS_OK) {
    state = PEPS_REQ_FAILED;
  } else {
    // small requests spend much of a step in host-side launch work: replay captured graphs
    // (batched engine only; the per-block engine launches one kernel per phase anyway)
    peps_set_graphs(ctx, 1);
    const peps_request& q = r->req;
    if (q.n_burn > 0 && peps_mc_sweep(ctx, q.n_burn, q.p1_until_beta > 0.0 ? 1 : 2) < 0)
      state = PEPS_REQ_FAILED;
    double t = 0;
    while (state == PEPS_REQ_DONE && t < q.t_end - 1e-12) {
      {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) {
          state = PEPS_REQ_CANCELLED;
          break;
        }
      }
      int p = (4.0 * t < q.p1_until_beta) ? 1 : 2;
      peps_stats stt{};
      auto t0 = Clock::now();
      int rc = peps_step(ctx, q.n_sweeps > 0 ? q.n_sweeps : 1, p, q.tau, q.eps, q.max_cg,
                         q.cg_tol, &stt);
      auto t1 = Clock::now();
      if (rc < 0) {
        state = PEPS_REQ_FAILED;
        break;
      }
      t += q.tau;
      double ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
      std::lock_guard<std::mutex> lk(s->mu);
      r->steps.push_back(stt);
      r->step_ms.push_back(ms);
      s->all_ms.push_back(ms);
      s->samples += P.n_chains;
      s->t_last = t1;
    }
    if (state == PEPS_REQ_DONE) {
      std::vector<double> th(peps_num_params(ctx));
      if (peps_get_theta(ctx, th.data(), th.size()) == PEPS_OK) {
        std::lock_guard<std::mutex> lk(s->mu);
        r->theta.swap(th);
      } else {
        state = PEPS_REQ_FAILED;
      }
    }
  }
  if (ctx) peps_free(ctx);
  if (st) cudaStreamDestroy(st);
  std::lock_guard<std::mutex> lk(s->mu);
  r->state = state;
  s->used -= r->footprint;
  s->active -= 1;
  admit(s);   // a slot and its memory are free: start the next queued requests
  s->cv.notify_all();
}

// Admits queued requests while they fit (caller holds the lock).
void admit(peps_server* s) {
  if (s->stopping) {
    for (int id : s->queue) s->reqs[id]->state = PEPS_REQ_CANCELLED;
    s->queue.clear();
    return;
  }
  while (!s->queue.empty() && s->active < s->max_active) {
    Request* r = s->reqs[s->queue.front()].get();
    if (s->used + r->footprint > s->budget) break;   // arrival order: wait for memory
    s->queue.pop_front();
    s->used += r->footprint;
    s->active += 1;
    r->state = PEPS_REQ_RUNNING;
    if (!s->started) {
      s->started = true;
      s->t_first = Clock::now();
    }
    r->worker = std::thread(run_request, s, r);
  }
}

}  // namespace

extern "C" {

int peps_srv_create(size_t budget, int max_active, int blocks, peps_server** out) {
  if (!out || max_active < 1 || blocks < 0) return PEPS_EINVAL;
  auto* s = new peps_server();
  cudaGetDevice(&s->device);
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete s;
      return PEPS_ECUDA;
    }
    budget = (size_t)(0.8 * (double)fr);
  }
  s->budget = budget;
  s->max_active = max_active;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
  s->blocks = blocks > 0 ? blocks : std::max(1, 4 * sms / max_active);
  *out = s;
  return PEPS_OK;
}

int peps_srv_submit(peps_server* s, const peps_request* q, int* id) {
  if (!s || !q || !id || !(q->tau > 0) || !(q->t_end >= 0) || q->max_cg < 0) return PEPS_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return PEPS_ESTATE;
  }
  peps_params P = q->params;
  if (s->blocks > 0 && P.n_blocks == 0) P.n_blocks = s->blocks;
  size_t fp = peps_footprint(&P);
  if (fp == 0 || fp > s->budget) return PEPS_EINVAL;
  auto r = std::make_unique<Request>();
  r->req = *q;
  r->footprint = fp;
  std::lock_guard<std::mutex> lk(s->mu);
  r->id = s->next_id++;
  *id = r->id;
  s->queue.push_back(r->id);
  s->reqs[r->id] = std::move(r);
  admit(s);
  return PEPS_OK;
}

int peps_srv_poll(peps_server* s, int id, int* state, int* n_steps, peps_stats* per, int cap) {
  if (!s) return PEPS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return PEPS_EINVAL;
  Request* r = it->second.get();
  if (state) *state = r->state;
  if (n_steps) *n_steps = (int)r->steps.size();
  if (per)
    for (int i = 0; i < cap && i < (int)r->steps.size(); ++i) per[i] = r->steps[i];
  return PEPS_OK;
}

int peps_srv_theta(peps_server* s, int id, double* host, size_t n) {
  if (!s || !host) return PEPS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end() || it->second->state != PEPS_REQ_DONE || it->second->theta.size() != n)
    return PEPS_EINVAL;
  std::copy(it->second->theta.begin(), it->second->theta.end(), host);
  return PEPS_OK;
}

int peps_srv_stop(peps_server* s) {
  if (!s) return PEPS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  s->stopping = true;
  admit(s);   // cancels what is still queued
  s->cv.notify_all();
  return PEPS_OK;
}

int peps_srv_drain(peps_server* s) {
  if (!s) return PEPS_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    admit(s);
    if (s->queue.empty() && s->active == 0) break;
    s->cv.wait(lk);
  }
  for (auto& kv : s->reqs)
    if (kv.second->worker.joinable()) kv.second->worker.join();
  for (auto& kv : s->reqs)
    if (kv.second->state == PEPS_REQ_FAILED) return PEPS_ECUDA;
  return PEPS_OK;
}

int peps_srv_metrics(peps_server* s, double* p50, double* p99, double* sps, int64_t* n) {
  if (!s) return PEPS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  std::vector<double> v = s->all_ms;
  std::sort(v.begin(), v.end());
  auto q = [&](double f) {
    if (v.empty()) return 0.0;
    size_t i = std::min(v.size() - 1, (size_t)(f * (double)v.size()));
    return v[i];
  };
  if (p50) *p50 = q(0.5);
  if (p99) *p99 = q(0.99);
  double secs = s->started ? std::chrono::duration<double>(s->t_last - s->t_first).count() : 0;
  if (sps) *sps = secs > 0 ? (double)s->samples / secs : 0;
  if (n) *n = (int64_t)v.size();
  return PEPS_OK;
}

void peps_srv_free(peps_server* s) {
  if (!s) return;
  peps_srv_drain(s);
  delete s;
}

}  // extern "C"
