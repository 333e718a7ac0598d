// Serving loop: continuous batching of filtered top-K requests over a resident
// index (appendix "Batch Inference" and "Memory Pre-Allocation": one scan
// serves a batch of queries, and every buffer is allocated up front).
//
// The server owns S slots.  A slot is a search context sharing the index's
// rows and term storage, with its own workspace, pinned staging, device
// output rows and CUDA stream; how many slots exist is decided by the memory
// the caller grants (arena_bytes / one slot's workspace).  A scheduler thread
// runs the loop:
//   * retire: a busy slot whose completion event has fired hands each of its
//     requests its rows of the batch result and becomes free;
//   * admit: a free slot takes pending requests first-come first-served while
//     the batch still fits the slot (queries <= the slot's batch capacity,
//     term occurrences <= its filter workspace), then launches one search on
//     its stream -- query upload, scan, selection and the result download are
//     all stream-ordered, so the thread never blocks on the GPU and searches of
//     different slots overlap on the device;
//   * requests that arrive while every slot is busy wait in the queue and join
//     the next batch that a slot forms (continuous batching).
// Latency is measured per request from submit to the moment its result is on
// the host.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "lr_internal.h"

namespace lr {
lr_status fail(lr_status st, const std::string &msg);  // runtime.cu: records the calling thread's error message
}

using namespace lr;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
  uint64_t ticket = 0;
  int B = 0, k_max = 0;
  std::vector<float> q;  // [B][dim]
  std::vector<int32_t> q_off, c_off, k;
  std::vector<uint32_t> terms;
  Clock::time_point t_submit;
  // result
  bool done = false;
  lr_status status = LR_OK;
  std::string message;  // the failure's message, recorded on the scheduler thread
  std::vector<int32_t> ids, count;  // [B][k_max], [B]
  std::vector<float> scores;
  double latency_ms = 0.0;
};

struct Slot {
  lr_index *ix = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  float *q_dev = nullptr;
  int32_t *ids_dev = nullptr, *cnt_dev = nullptr;
  float *sc_dev = nullptr;
  float *q_h = nullptr;
  int32_t *ids_h = nullptr, *cnt_h = nullptr;
  float *sc_h = nullptr;
  std::vector<Request *> reqs;
  int B = 0, k_all = 0;
  bool busy = false;
  lr_status launch_status = LR_OK;
  std::string launch_message;
};

}  // namespace

struct lr_server {
  lr_index *base = nullptr;
  int device = 0, dim = 0, vocab = 0, max_q = 0, max_k = 0, max_terms = 0;
  size_t slot_bytes = 0;
  lr_search_opts opts{};
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request *> pending;
  std::unordered_map<uint64_t, Request *> live;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread th;
  // statistics
  std::vector<double> lat;
  int64_t submitted = 0, completed = 0, batches = 0, queries = 0;
  Clock::time_point t0;
};

namespace {

lr_status validate_request(const lr_server *S, int B, const lr_filters *f, const int32_t *k, int k_all) {
  if (B < 1) return fail(LR_ERR_INVALID, "request: B must be >= 1");
  if (B > S->max_q) return fail(LR_ERR_WORKSPACE, "request: more queries than a serving slot holds");
  if (!f || !f->q_off) return fail(LR_ERR_INVALID, "request: null filters");
  if (f->q_off[0] != 0) return fail(LR_ERR_INVALID, "request: q_off[0] must be 0");
  for (int b = 0; b < B; ++b)
    if (f->q_off[b + 1] < f->q_off[b]) return fail(LR_ERR_INVALID, "request: q_off must be non-decreasing");
  const int nC = f->q_off[B];
  if (nC > 0 && (!f->c_off || !f->terms)) return fail(LR_ERR_INVALID, "request: null clause arrays");
  if (nC > 0 && f->c_off[0] != 0) return fail(LR_ERR_INVALID, "request: c_off[0] must be 0");
  for (int c = 0; c < nC; ++c)
    if (f->c_off[c + 1] <= f->c_off[c]) return fail(LR_ERR_INVALID, "request: a clause with zero terms");
  const int nT = nC > 0 ? f->c_off[nC] : 0;
  if (nT > S->max_terms) return fail(LR_ERR_WORKSPACE, "request: more term occurrences than a slot holds");
  for (int i = 0; i < nT; ++i)
    if (f->terms[i] >= (uint32_t)S->vocab) return fail(LR_ERR_INVALID, "request: term id >= vocab");
  for (int b = 0; b < B; ++b) {
    const int kb = k ? k[b] : k_all;
    if (kb < 1 || kb > S->max_k || kb > k_all) return fail(LR_ERR_INVALID, "request: K out of range");
  }
  return LR_OK;
}

// Launch one batch on a free slot (called without the lock; the slot's
// requests are owned by the scheduler thread until the slot is retired).
void launch(lr_server *S, Slot &sl) {
  int B = 0, k_all = 0;
  std::vector<int32_t> q_off{0}, c_off{0}, k;
  std::vector<uint32_t> terms;
  for (Request *r : sl.reqs) {
    std::memcpy(sl.q_h + (size_t)B * S->dim, r->q.data(), sizeof(float) * r->q.size());
    const int cbase = (int)c_off.size() - 1;
    const int tbase = (int)terms.size();
    for (int b = 0; b < r->B; ++b) q_off.push_back(cbase + r->q_off[b + 1]);
    for (size_t c = 1; c < r->c_off.size(); ++c) c_off.push_back(tbase + r->c_off[c]);
    terms.insert(terms.end(), r->terms.begin(), r->terms.end());
    k.insert(k.end(), r->k.begin(), r->k.end());
    k_all = std::max(k_all, r->k_max);
    B += r->B;
  }
  if (terms.empty()) terms.push_back(0);
  sl.B = B;
  sl.k_all = k_all;
  lr_filters f{q_off.data(), c_off.data(), terms.data()};
  lr_status st = LR_OK;
  if (cudaMemcpyAsync(sl.q_dev, sl.q_h, sizeof(float) * (size_t)B * S->dim, cudaMemcpyHostToDevice, sl.stream) !=
      cudaSuccess)
    st = fail(LR_ERR_CUDA, "serving: query upload failed");
  if (st == LR_OK)
    st = lr_search_ex(sl.ix, sl.q_dev, B, &f, k.data(), k_all, sl.ids_dev, sl.sc_dev, sl.cnt_dev, &S->opts, nullptr,
                      sl.stream);
  if (st == LR_OK) {
    const size_t n = (size_t)B * k_all;
    if (cudaMemcpyAsync(sl.ids_h, sl.ids_dev, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, sl.stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(sl.sc_h, sl.sc_dev, sizeof(float) * n, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess ||
        cudaMemcpyAsync(sl.cnt_h, sl.cnt_dev, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, sl.stream) !=
            cudaSuccess)
      st = fail(LR_ERR_CUDA, "serving: result download failed");
  }
  if (cudaEventRecord(sl.done, sl.stream) != cudaSuccess) st = fail(LR_ERR_CUDA, "serving: event record failed");
  sl.launch_status = st;
  sl.launch_message = st == LR_OK ? std::string() : std::string(lr_last_error_message());
}

// Hand each request of a finished slot its rows (called with the lock held).
void retire(lr_server *S, Slot &sl) {
  const Clock::time_point now = Clock::now();
  int row = 0;
  for (Request *r : sl.reqs) {
    r->status = sl.launch_status;
    r->message = sl.launch_message;
    r->ids.assign((size_t)r->B * r->k_max, -1);
    r->scores.assign((size_t)r->B * r->k_max, -INFINITY);
    r->count.assign(r->B, 0);
    if (r->status == LR_OK) {
      for (int b = 0; b < r->B; ++b, ++row) {
        std::memcpy(&r->ids[(size_t)b * r->k_max], sl.ids_h + (size_t)row * sl.k_all, sizeof(int32_t) * r->k_max);
        std::memcpy(&r->scores[(size_t)b * r->k_max], sl.sc_h + (size_t)row * sl.k_all, sizeof(float) * r->k_max);
        r->count[b] = sl.cnt_h[row];
      }
    }
    r->latency_ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
    r->done = true;
    S->lat.push_back(r->latency_ms);
    ++S->completed;
  }
  ++S->batches;
  S->queries += sl.B;
  sl.reqs.clear();
  sl.busy = false;
  S->cv_done.notify_all();
}

void scheduler(lr_server *S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    bool busy = false;
    for (Slot &sl : S->slots) {
      if (!sl.busy) continue;
      const cudaError_t e = cudaEventQuery(sl.done);
      if (e == cudaSuccess) {
        retire(S, sl);
      } else {
        if (e == cudaErrorNotReady) cudaGetLastError();  // not an error: the batch is still running
        busy = true;
      }
    }
    for (Slot &sl : S->slots) {
      if (sl.busy || S->pending.empty()) continue;
      // admission: first come first served while the batch fits the slot
      int nq = 0, nt = 0;
      while (!S->pending.empty()) {
        Request *r = S->pending.front();
        const int rt = (int)r->terms.size();
        if (nq + r->B > S->max_q || nt + rt > S->max_terms) break;
        nq += r->B;
        nt += rt;
        sl.reqs.push_back(r);
        S->pending.pop_front();
      }
      sl.busy = true;
      busy = true;
      lk.unlock();
      launch(S, sl);
      lk.lock();
    }
    if (S->stop && S->pending.empty() && !busy) break;
    if (busy) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    } else {
      S->cv_work.wait(lk, [&] { return S->stop || !S->pending.empty(); });
    }
  }
}

void free_slot(Slot &sl) {
  if (sl.stream) cudaStreamSynchronize(sl.stream);
  index_destroy_slot(sl.ix);
  cudaFree(sl.q_dev);
  cudaFree(sl.ids_dev);
  cudaFree(sl.sc_dev);
  cudaFree(sl.cnt_dev);
  cudaFreeHost(sl.q_h);
  cudaFreeHost(sl.ids_h);
  cudaFreeHost(sl.sc_h);
  cudaFreeHost(sl.cnt_h);
  if (sl.done) cudaEventDestroy(sl.done);
  if (sl.stream) cudaStreamDestroy(sl.stream);
}

}  // namespace

extern "C" {

lr_status lr_server_create(lr_index *index, const lr_server_opts *opts, size_t arena_bytes, lr_server **out) {
  if (!index || !opts || !out) return fail(LR_ERR_INVALID, "lr_server_create: null argument");
  *out = nullptr;
  if (opts->slots < 1 || opts->max_queries < 1) return fail(LR_ERR_INVALID, "slots and max_queries must be >= 1");
  lr_server *S = new lr_server();
  S->base = index;
  S->device = index_device(index);
  S->dim = index_dim(index);
  S->vocab = index_vocab(index);
  S->max_q = opts->max_queries;
  S->max_k = index_max_k(index);
  S->max_terms = 16 * opts->max_queries + 64;
  S->opts.plan = opts->plan;
  cudaSetDevice(S->device);
  for (int i = 0; i < opts->slots; ++i) {
    Slot sl;
    lr_status st = index_clone_slot(index, S->max_q, nullptr, &sl.ix);
    if (st != LR_OK) {
      if (i == 0) {
        delete S;
        return st;
      }
      break;  // fewer slots than asked: the device memory is used up
    }
    const size_t rows = (size_t)S->max_q * S->max_k;
    const bool ok = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess &&
                    cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess &&
                    cudaMalloc(&sl.q_dev, sizeof(float) * S->max_q * S->dim) == cudaSuccess &&
                    cudaMalloc(&sl.ids_dev, sizeof(int32_t) * rows) == cudaSuccess &&
                    cudaMalloc(&sl.sc_dev, sizeof(float) * rows) == cudaSuccess &&
                    cudaMalloc(&sl.cnt_dev, sizeof(int32_t) * S->max_q) == cudaSuccess &&
                    cudaHostAlloc((void **)&sl.q_h, sizeof(float) * S->max_q * S->dim, 0) == cudaSuccess &&
                    cudaHostAlloc((void **)&sl.ids_h, sizeof(int32_t) * rows, 0) == cudaSuccess &&
                    cudaHostAlloc((void **)&sl.sc_h, sizeof(float) * rows, 0) == cudaSuccess &&
                    cudaHostAlloc((void **)&sl.cnt_h, sizeof(int32_t) * S->max_q, 0) == cudaSuccess;
    const size_t bytes = lr_index_device_bytes(sl.ix) + sizeof(float) * S->max_q * S->dim + 8 * rows + 4 * S->max_q;
    if (i == 0) S->slot_bytes = bytes;
    if (!ok) {
      cudaGetLastError();
      free_slot(sl);
      if (i == 0) {
        delete S;
        return fail(LR_ERR_NOMEM, "cannot allocate a serving slot");
      }
      break;
    }
    if (i == 0) S->max_terms = index_max_batch_terms(sl.ix);  // the slot's filter workspace
    S->slots.push_back(sl);
    // memory-based admission of slots: stop when the next slot would exceed the arena
    if (arena_bytes > 0 && (size_t)(i + 2) * S->slot_bytes > arena_bytes) break;
  }
  S->t0 = Clock::now();
  S->th = std::thread(scheduler, S);
  *out = S;
  return LR_OK;
}

lr_status lr_server_submit(lr_server *S, const float *q, int32_t B, const lr_filters *f, const int32_t *k,
                           int32_t k_all, uint64_t *ticket) {
  if (!S || !q || !ticket) return fail(LR_ERR_INVALID, "lr_server_submit: null argument");
  lr_status st = validate_request(S, B, f, k, k_all);
  if (st != LR_OK) return st;
  Request *r = new Request();
  r->B = B;
  r->q.assign(q, q + (size_t)B * S->dim);
  r->q_off.assign(f->q_off, f->q_off + B + 1);
  const int nC = f->q_off[B];
  r->c_off.assign(f->c_off ? f->c_off : nullptr, f->c_off ? f->c_off + nC + 1 : nullptr);
  if (r->c_off.empty()) r->c_off.push_back(0);
  const int nT = r->c_off.back();
  if (nT > 0) r->terms.assign(f->terms, f->terms + nT);
  r->k.resize(B);
  int km = 0;
  for (int b = 0; b < B; ++b) {
    r->k[b] = k ? k[b] : k_all;
    km = std::max(km, r->k[b]);
  }
  r->k_max = km;
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) {
      delete r;
      return fail(LR_ERR_INVALID, "server is shutting down");
    }
    r->ticket = S->next_ticket++;
    S->live[r->ticket] = r;
    S->pending.push_back(r);
    ++S->submitted;
    *ticket = r->ticket;
  }
  S->cv_work.notify_one();
  return LR_OK;
}

lr_status lr_server_wait(lr_server *S, uint64_t ticket, int32_t timeout_ms, int32_t *out_ids, float *out_scores,
                         int32_t *out_count, int32_t k_stride, double *latency_ms) {
  if (!S) return fail(LR_ERR_INVALID, "lr_server_wait: null server");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->live.find(ticket);
  if (it == S->live.end()) return fail(LR_ERR_INVALID, "lr_server_wait: unknown ticket");
  Request *r = it->second;
  const bool got = S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 1 << 30 : timeout_ms),
                                       [&] { return r->done; });
  if (!got) return fail(LR_ERR_TIMEOUT, "lr_server_wait: request not finished in time");
  if (k_stride < r->k_max) return fail(LR_ERR_INVALID, "lr_server_wait: k_stride below the request's K");
  for (int b = 0; b < r->B; ++b) {
    for (int i = 0; i < k_stride; ++i) {
      const bool in = i < r->k_max;
      if (out_ids) out_ids[(size_t)b * k_stride + i] = in ? r->ids[(size_t)b * r->k_max + i] : -1;
      if (out_scores) out_scores[(size_t)b * k_stride + i] = in ? r->scores[(size_t)b * r->k_max + i] : -INFINITY;
    }
    if (out_count) out_count[b] = r->count[b];
  }
  if (latency_ms) *latency_ms = r->latency_ms;
  const lr_status st = r->status;
  const std::string msg = r->message;
  S->live.erase(it);
  delete r;
  return st == LR_OK ? LR_OK : fail(st, "request failed: " + msg);
}

lr_status lr_server_get_stats(lr_server *S, lr_server_stats *st, int32_t reset) {
  if (!S || !st) return fail(LR_ERR_INVALID, "lr_server_get_stats: null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  std::vector<double> v = S->lat;
  std::sort(v.begin(), v.end());
  auto pct = [&](double p) { return v.empty() ? 0.0 : v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
  double mean = 0.0;
  for (double x : v) mean += x;
  st->submitted = S->submitted;
  st->completed = S->completed;
  st->batches = S->batches;
  st->queries = S->queries;
  st->slots = (int32_t)S->slots.size();
  st->slot_bytes = S->slot_bytes;
  st->p50_ms = pct(0.50);
  st->p99_ms = pct(0.99);
  st->mean_ms = v.empty() ? 0.0 : mean / v.size();
  st->max_ms = v.empty() ? 0.0 : v.back();
  st->elapsed_s = std::chrono::duration<double>(Clock::now() - S->t0).count();
  if (reset) {
    S->lat.clear();
    S->submitted = S->completed = S->batches = S->queries = 0;
    S->t0 = Clock::now();
  }
  return LR_OK;
}

lr_status lr_server_destroy(lr_server *S) {
  if (!S) return LR_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->th.joinable()) S->th.join();
  cudaSetDevice(S->device);
  for (Slot &sl : S->slots) free_slot(sl);
  for (auto &kv : S->live) delete kv.second;
  delete S;
  return LR_OK;
}

}  // extern "C"
