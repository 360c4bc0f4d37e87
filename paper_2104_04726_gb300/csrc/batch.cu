// Batched and served forms of the stack pipeline (host runtime).
//
// A problem is the colour pre-pass, the Tucker-ALS decomposition of
// Section III-B and the core quantiser of one stack, enqueued on one stream
// by the same entry points a single call uses, so its result does not depend
// on what else runs.  The batch context deals many problems to a pool of
// streams (longest first, to the least-loaded stream) and can capture the
// whole enqueue into one CUDA graph.  The server admits problems from a
// queue into a fixed set of slots under a device-memory budget, from its
// own host thread, and keeps per-request latency.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <future>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace {

// Validation plus the device memory the problem's workspace takes.
mes_status problem_check(const mes_problem& p, size_t* ws_bytes) {
  if (p.N < 2 || p.N > 8) return mes::fail(MES_ERR_INVALID_ARG, "problem: N must be 2..8");
  if (!p.X || !p.core) return mes::fail(MES_ERR_INVALID_ARG, "problem: null X or core");
  for (int n = 0; n < p.N; ++n)
    if (!p.factors[n]) return mes::fail(MES_ERR_INVALID_ARG, "problem: factors[%d] is null", n);
  if (p.rgb8) {
    if (p.N != 4 || p.dims[2] != 3)
      return mes::fail(MES_ERR_INVALID_ARG, "problem: 8-bit input needs dims (s1, s2, 3, K)");
    if (p.space != MES_YCBCR601 && p.space != MES_IPT && p.space != MES_YCBCR2020CL)
      return mes::fail(MES_ERR_INVALID_ARG, "problem: unknown colour space %d", p.space);
    if (p.gamma < 0.f) return mes::fail(MES_ERR_INVALID_ARG, "problem: gamma must be >= 0");
  }
  if (p.quant_bits != 0) {
    if (p.quant_bits < 2 || p.quant_bits > 16)
      return mes::fail(MES_ERR_INVALID_ARG, "problem: quant_bits must be 0 or 2..16");
    if (!p.q || !p.scales) return mes::fail(MES_ERR_INVALID_ARG, "problem: null q or scales");
  }
  if (p.max_iters < 1) return mes::fail(MES_ERR_INVALID_ARG, "problem: max_iters must be >= 1");
  size_t ws = 0;
  MES_TRY(mes_tucker_als_workspace_size(p.N, p.dims, p.ranks, &p.opts, &ws));
  int64_t planes = 1;
  for (int n = 2; n < p.N; ++n) planes *= p.ranks[n];
  // colour norm partials and the quantiser's per-plane words
  ws += 64 * 1024 + (size_t)planes * 16;
  if (ws_bytes) *ws_bytes = ws;
  return MES_OK;
}

// Device bytes the caller's buffers of the problem occupy.
size_t problem_io_bytes(const mes_problem& p) {
  int64_t nX = 1, nQ = 1, nf = 0, planes = 1;
  for (int n = 0; n < p.N; ++n) {
    nX *= p.dims[n];
    nQ *= p.ranks[n];
    nf += p.dims[n] * p.ranks[n];
  }
  for (int n = 2; n < p.N; ++n) planes *= p.ranks[n];
  size_t b = (size_t)(nX + nQ + nf) * 4 + 8;
  if (p.rgb8) b += (size_t)nX;
  if (p.quant_bits) b += (size_t)nQ * 2 + (size_t)planes * 4;
  return b;
}

// Work estimate for ordering: the two large contractions of every sweep.
double problem_cost(const mes_problem& p) {
  double L = 1;
  for (int n = 2; n < p.N; ++n) L *= (double)p.dims[n];
  return (double)p.max_iters * (double)p.dims[0] * (double)p.dims[1] * L * (double)(p.ranks[0] + p.ranks[1]) +
         (double)p.dims[0] * (double)p.dims[1] * L;
}

mes_status problem_enqueue(const mes_problem& p, cudaStream_t st) {
  void* s = static_cast<void*>(st);
  if (p.rgb8)
    MES_TRY(mes_colour_convert(p.rgb8, p.dims[0], p.dims[1], p.dims[3], p.space,
                               p.gamma > 0.f ? p.gamma : 2.2f, p.X, nullptr, s));
  MES_TRY(mes_tucker_als(p.X, p.N, p.dims, p.ranks, p.max_iters, p.tol, p.core, p.factors, p.fit, &p.opts, s));
  if (p.quant_bits) MES_TRY(mes_quantize_core(p.core, p.N, p.ranks, p.quant_bits, p.q, p.scales, 0, s));
  return MES_OK;
}

}  // namespace

// --------------------------------------------------------------------------
// batch
// --------------------------------------------------------------------------
struct mes_batch {
  int device = 0;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

mes_status batch_enqueue(mes_batch* b, const mes_problem* probs, int n, mes_status* statuses,
                         cudaStream_t stream) {
  if (!b || !probs || n < 1) return mes::fail(MES_ERR_INVALID_ARG, "mes_batch: null handle/problems or n < 1");
  std::vector<double> cost(n);
  mes_status first = MES_OK;
  for (int i = 0; i < n; ++i) {
    mes_status s = problem_check(probs[i], nullptr);
    if (statuses) statuses[i] = s;
    if (s != MES_OK && first == MES_OK) first = s;
    cost[i] = problem_cost(probs[i]);
  }
  if (first != MES_OK) return first;
  // longest first, each to the stream with the least work so far
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
  const int ns = std::min<int>((int)b->streams.size(), n);
  std::vector<double> load(ns, 0.0);
  MES_CUDA_TRY(cudaEventRecord(b->fork, stream));
  for (int k = 0; k < ns; ++k) MES_CUDA_TRY(cudaStreamWaitEvent(b->streams[k], b->fork, 0));
  mes_status err = MES_OK;
  for (int i : order) {
    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[k] += cost[i];
    mes_problem pi = probs[i];
    if (pi.opts.concurrency == 0) pi.opts.concurrency = ns;   // the streams running side by side
    mes_status s = problem_enqueue(pi, b->streams[k]);
    if (statuses) statuses[i] = s;
    if (s != MES_OK) {
      err = s;
      break;
    }
  }
  // join every forked stream back, also after an error, so `stream` (or a
  // capture) never holds unjoined work
  for (int k = 0; k < ns; ++k) {
    MES_CUDA_TRY(cudaEventRecord(b->joins[k], b->streams[k]));
    MES_CUDA_TRY(cudaStreamWaitEvent(stream, b->joins[k], 0));
  }
  return err;
}

}  // namespace

extern "C" mes_status mes_batch_create(int max_streams, mes_batch** out) {
  mes::clear_error();
  if (!out) return mes::fail(MES_ERR_INVALID_ARG, "mes_batch_create: null out");
  *out = nullptr;
  if (max_streams < 1 || max_streams > 64)
    return mes::fail(MES_ERR_INVALID_ARG, "mes_batch_create: max_streams must be 1..64");
  mes_batch* b = new mes_batch();
  cudaGetDevice(&b->device);
  mes_status st = MES_OK;
  auto chk = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && st == MES_OK) {
      cudaGetLastError();
      st = mes::fail(MES_ERR_CUDA, "mes_batch_create: %s: %s", what, cudaGetErrorString(e));
    }
  };
  chk(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "cudaEventCreate");
  for (int k = 0; k < max_streams && st == MES_OK; ++k) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    chk(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "cudaStreamCreate");
    chk(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
    if (s) b->streams.push_back(s);
    if (e) b->joins.push_back(e);
  }
  if (st != MES_OK) {
    for (cudaStream_t x : b->streams) cudaStreamDestroy(x);
    for (cudaEvent_t x : b->joins) cudaEventDestroy(x);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
    return st;
  }
  *out = b;
  return MES_OK;
}

extern "C" mes_status mes_batch_run(mes_batch* b, const mes_problem* probs, int n, mes_status* statuses,
                                    void* stream) {
  mes::clear_error();
  return batch_enqueue(b, probs, n, statuses, static_cast<cudaStream_t>(stream));
}

extern "C" mes_status mes_batch_capture(mes_batch* b, const mes_problem* probs, int n, void* stream) {
  mes::clear_error();
  if (!b) return mes::fail(MES_ERR_INVALID_ARG, "mes_batch_capture: null handle");
  if (mes::prof_on()) return mes::fail(MES_ERR_INVALID_ARG, "mes_batch_capture: kernel profiler is on");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!st) return mes::fail(MES_ERR_INVALID_ARG, "mes_batch_capture: the legacy stream cannot be captured");
  MES_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
  mes_status s = batch_enqueue(b, probs, n, nullptr, st);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &graph);
  if (s != MES_OK) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return s;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return mes::fail(MES_ERR_CUDA, "mes_batch_capture: cudaStreamEndCapture: %s", cudaGetErrorString(e));
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return mes::fail(MES_ERR_CUDA, "mes_batch_capture: cudaGraphInstantiate: %s", cudaGetErrorString(e));
  }
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = exec;
  return MES_OK;
}

extern "C" mes_status mes_batch_launch(mes_batch* b, void* stream) {
  mes::clear_error();
  if (!b || !b->exec) return mes::fail(MES_ERR_INVALID_ARG, "mes_batch_launch: nothing captured");
  MES_CUDA_TRY(cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)));
  return MES_OK;
}

extern "C" mes_status mes_batch_destroy(mes_batch* b) {
  mes::clear_error();
  if (!b) return MES_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  for (cudaStream_t s : b->streams) cudaStreamSynchronize(s);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  cudaSetDevice(prev);
  cudaGetLastError();
  delete b;
  return MES_OK;
}

// --------------------------------------------------------------------------
// server
// --------------------------------------------------------------------------
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  mes_problem p;
  size_t bytes = 0;
  Clock::time_point submitted;
  int slot = -1;
  bool done = false;
  mes_status status = MES_OK;
  double latency_ms = 0.0;
};

}  // namespace

struct mes_server {
  int device = 0;
  size_t budget = 0;
  std::vector<cudaStream_t> slots;
  std::vector<cudaEvent_t> slot_done;
  std::vector<uint64_t> slot_req;   // 0 = free
  // per slot: the device-side status word of the running decomposition
  // (used when the request brings none) and its pinned host copy, read once
  // the slot's completion event has fired
  int* dev_status = nullptr;
  int* host_status = nullptr;
  // per slot: the host task enqueueing the admitted request (its launches
  // are issued off the admission thread, so admission and retirement go on
  // while a large request is being enqueued)
  std::vector<std::future<mes_status>> slot_enq;
  std::vector<char> slot_enqueuing;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Request> reqs;
  uint64_t next_id = 1;
  size_t in_use = 0, peak = 0;
  uint64_t submitted = 0, completed = 0, failed = 0;
  std::vector<double> latencies;
  Clock::time_point t0;
  double first_admit = -1.0, last_done = -1.0;
  bool stop = false;
  std::thread worker;
};

namespace {

double secs(Clock::time_point a, Clock::time_point b) { return std::chrono::duration<double>(b - a).count(); }

// The loop: retire finished slots, then admit from the queue in order
// (a request that does not fit lets up to max_slots later ones pass).
void serve_loop(mes_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    bool progressed = false;
    // retire
    for (size_t k = 0; k < s->slots.size(); ++k) {
      const uint64_t id = s->slot_req[k];
      if (!id) continue;
      mes_status enq = MES_OK;
      if (s->slot_enqueuing[k]) {
        // still enqueueing, or just done: the task's status decides
        if (s->slot_enq[k].wait_for(std::chrono::seconds(0)) != std::future_status::ready) continue;
        enq = s->slot_enq[k].get();
        s->slot_enqueuing[k] = 0;
      }
      cudaError_t q = cudaSuccess;
      if (enq == MES_OK) {
        q = cudaEventQuery(s->slot_done[k]);
        if (q == cudaErrorNotReady) continue;
      }
      Request& r = s->reqs[id];
      r.done = true;
      if (enq != MES_OK) {
        r.status = enq;
      } else if (q != cudaSuccess) {
        cudaGetLastError();
        r.status = MES_ERR_CUDA;
      } else if (s->host_status[k] != MES_OK) {
        r.status = static_cast<mes_status>(s->host_status[k]);   // failure met on the device
      }
      const auto now = Clock::now();
      r.latency_ms = 1e3 * secs(r.submitted, now);
      s->last_done = secs(s->t0, now);
      s->in_use -= r.bytes;
      s->slot_req[k] = 0;
      if (r.status == MES_OK) {
        ++s->completed;
        s->latencies.push_back(r.latency_ms);
      } else {
        ++s->failed;
      }
      progressed = true;
    }
    if (progressed) s->cv_done.notify_all();
    // admit: the first queued request (within a window of max_slots passes)
    // that fits next to the running ones goes to a free slot; the lock is
    // released while its work is enqueued
    while (true) {
      int k = -1;
      for (size_t j = 0; j < s->slots.size(); ++j)
        if (!s->slot_req[j]) {
          k = (int)j;
          break;
        }
      if (k < 0) break;
      auto it = s->queue.begin();
      int passed = 0;
      for (; it != s->queue.end() && passed <= (int)s->slots.size(); ++it, ++passed)
        if (s->in_use + s->reqs[*it].bytes <= s->budget) break;
      if (it == s->queue.end() || passed > (int)s->slots.size()) break;
      const uint64_t id = *it;
      s->queue.erase(it);
      Request& r = s->reqs[id];   // node-based map: the reference stays valid
      if (mes::fault_admit()) {
        // injected refusal: the request ends without running
        r.done = true;
        r.status = MES_ERR_OOM;
        r.latency_ms = 1e3 * secs(r.submitted, Clock::now());
        ++s->failed;
        s->cv_done.notify_all();
        progressed = true;
        continue;
      }
      s->slot_req[k] = id;
      s->in_use += r.bytes;
      s->peak = std::max(s->peak, s->in_use);
      r.slot = k;
      mes_problem prob = r.p;
      if (prob.opts.concurrency == 0) prob.opts.concurrency = (int)s->slots.size();
      int* dstat = prob.opts.status ? prob.opts.status : s->dev_status + k;
      prob.opts.status = dstat;
      s->host_status[k] = MES_OK;
      if (s->first_admit < 0) s->first_admit = secs(s->t0, Clock::now());
      // the request's launches go out from a task of its own; the slot's
      // completion event is recorded after them, and the retirement above
      // reads it only once the task has finished
      const int dev = s->device;
      cudaStream_t sk = s->slots[k];
      int* hstat = s->host_status + k;
      cudaEvent_t done_ev = s->slot_done[k];
      s->slot_enqueuing[k] = 1;
      s->slot_enq[k] = std::async(std::launch::async, [prob, dev, sk, hstat, dstat, done_ev]() -> mes_status {
        cudaSetDevice(dev);
        mes_status st = problem_enqueue(prob, sk);
        if (st == MES_OK && (cudaMemcpyAsync(hstat, dstat, sizeof(int), cudaMemcpyDeviceToHost, sk) != cudaSuccess ||
                             cudaEventRecord(done_ev, sk) != cudaSuccess)) {
          cudaGetLastError();
          st = MES_ERR_CUDA;
        }
        if (st != MES_OK) cudaStreamSynchronize(sk);   // let what was enqueued finish
        return st;
      });
      progressed = true;
    }
    bool running = false;
    for (uint64_t id : s->slot_req) running |= (id != 0);
    if (s->stop && s->queue.empty() && !running) break;
    if (!progressed) {
      // poll running work at a short interval, sleep on the queue otherwise
      if (running)
        s->cv_work.wait_for(lk, std::chrono::microseconds(50));
      else
        s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
    }
  }
}

}  // namespace

extern "C" mes_status mes_serve_create(size_t hbm_budget_bytes, int max_slots, mes_server** out) {
  mes::clear_error();
  if (!out) return mes::fail(MES_ERR_INVALID_ARG, "mes_serve_create: null out");
  *out = nullptr;
  if (hbm_budget_bytes == 0) return mes::fail(MES_ERR_INVALID_ARG, "mes_serve_create: zero budget");
  if (max_slots < 1 || max_slots > 64)
    return mes::fail(MES_ERR_INVALID_ARG, "mes_serve_create: max_slots must be 1..64");
  mes_server* s = new mes_server();
  cudaGetDevice(&s->device);
  s->budget = hbm_budget_bytes;
  s->t0 = Clock::now();
  for (int k = 0; k < max_slots; ++k) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    cudaError_t e1 = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    cudaError_t e2 = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (st) s->slots.push_back(st);
    if (ev) s->slot_done.push_back(ev);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
      cudaGetLastError();
      for (cudaStream_t x : s->slots) cudaStreamDestroy(x);
      for (cudaEvent_t x : s->slot_done) cudaEventDestroy(x);
      delete s;
      return mes::fail(MES_ERR_CUDA, "mes_serve_create: stream or event creation failed");
    }
    s->slot_req.push_back(0);
  }
  // status words, allocated once here (never while serving)
  if (cudaMalloc(&s->dev_status, sizeof(int) * max_slots) != cudaSuccess ||
      cudaMallocHost(&s->host_status, sizeof(int) * max_slots) != cudaSuccess) {
    cudaGetLastError();
    if (s->dev_status) cudaFree(s->dev_status);
    for (cudaStream_t x : s->slots) cudaStreamDestroy(x);
    for (cudaEvent_t x : s->slot_done) cudaEventDestroy(x);
    delete s;
    return mes::fail(MES_ERR_OOM, "mes_serve_create: status words could not be allocated");
  }
  for (int k = 0; k < max_slots; ++k) s->host_status[k] = MES_OK;
  s->slot_enq.resize(max_slots);
  s->slot_enqueuing.assign(max_slots, 0);
  s->worker = std::thread(serve_loop, s);
  *out = s;
  return MES_OK;
}

extern "C" mes_status mes_serve_submit(mes_server* s, const mes_problem* p, uint64_t* ticket) {
  mes::clear_error();
  if (!s || !p || !ticket) return mes::fail(MES_ERR_INVALID_ARG, "mes_serve_submit: null argument");
  size_t ws = 0;
  MES_TRY(problem_check(*p, &ws));
  const size_t bytes = ws + problem_io_bytes(*p);
  if (bytes > s->budget)
    return mes::fail(MES_ERR_OOM, "mes_serve_submit: request needs %zu bytes, budget %zu", bytes, s->budget);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return mes::fail(MES_ERR_INVALID_ARG, "mes_serve_submit: server is stopping");
    Request r;
    r.id = s->next_id++;
    r.p = *p;
    r.bytes = bytes;
    r.submitted = Clock::now();
    s->reqs[r.id] = r;
    s->queue.push_back(r.id);
    ++s->submitted;
    *ticket = r.id;
  }
  s->cv_work.notify_one();
  return MES_OK;
}

extern "C" mes_status mes_serve_poll(mes_server* s, uint64_t ticket, int* done, mes_status* result,
                                     double* latency_ms) {
  mes::clear_error();
  if (!s || !done) return mes::fail(MES_ERR_INVALID_ARG, "mes_serve_poll: null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return mes::fail(MES_ERR_INVALID_ARG, "mes_serve_poll: unknown ticket");
  *done = it->second.done ? 1 : 0;
  if (it->second.done) {
    if (result) *result = it->second.status;
    if (latency_ms) *latency_ms = it->second.latency_ms;
  }
  return MES_OK;
}

extern "C" mes_status mes_serve_wait(mes_server* s, uint64_t ticket, double timeout_ms, mes_status* result,
                                     double* latency_ms) {
  mes::clear_error();
  if (!s) return mes::fail(MES_ERR_INVALID_ARG, "mes_serve_wait: null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return mes::fail(MES_ERR_INVALID_ARG, "mes_serve_wait: unknown ticket");
  const auto deadline = Clock::now() + std::chrono::microseconds((int64_t)(timeout_ms * 1e3));
  while (!s->reqs[ticket].done) {
    if (timeout_ms < 0) {
      s->cv_done.wait(lk);
    } else if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !s->reqs[ticket].done) {
      return mes::fail(MES_ERR_TIMEOUT, "mes_serve_wait: ticket %llu not done after %.1f ms",
                       (unsigned long long)ticket, timeout_ms);
    }
  }
  const Request& r = s->reqs[ticket];
  if (result) *result = r.status;
  if (latency_ms) *latency_ms = r.latency_ms;
  return MES_OK;
}

extern "C" mes_status mes_serve_get_stats(mes_server* s, mes_serve_stats* out) {
  mes::clear_error();
  if (!s || !out) return mes::fail(MES_ERR_INVALID_ARG, "mes_serve_get_stats: null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->queued = s->queue.size();
  for (uint64_t id : s->slot_req) out->running += (id != 0);
  std::vector<double> l = s->latencies;
  if (!l.empty()) {
    std::sort(l.begin(), l.end());
    // nearest-rank percentiles
    auto pct = [&](double q) {
      size_t i = (size_t)std::ceil(q * (double)l.size());
      if (i < 1) i = 1;
      return l[std::min(i, l.size()) - 1];
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = l.back();
    double sum = 0;
    for (double v : l) sum += v;
    out->mean_ms = sum / (double)l.size();
  }
  out->first_admit_s = s->first_admit;
  out->last_done_s = s->last_done;
  out->hbm_in_use = s->in_use;
  out->hbm_peak = s->peak;
  return MES_OK;
}

extern "C" mes_status mes_serve_destroy(mes_server* s) {
  mes::clear_error();
  if (!s) return MES_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  for (cudaStream_t x : s->slots) cudaStreamDestroy(x);
  for (cudaEvent_t x : s->slot_done) cudaEventDestroy(x);
  if (s->dev_status) cudaFree(s->dev_status);
  if (s->host_status) cudaFreeHost(s->host_status);
  cudaSetDevice(prev);
  cudaGetLastError();
  delete s;
  return MES_OK;
}
