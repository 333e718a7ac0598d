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
//
// With chunks = C >= 2 the server runs the rotating scan instead (Sec. 5.3's
// batch inference with requests joining a scan in flight): the index is cut
// into C row chunks, and every step scans one chunk for all active queries --
// one search restricted to the chunk's rows (lr_search_opts row range), whose
// per-query top K is merged on the device into the query's running top K
// (exact: the chunks hold disjoint rows and every list is ordered by (score
// desc, id asc)).  A query occupies a lane from admission until it has seen
// all C chunks, starting at whichever chunk comes next, so a request waits at
// most one step to start; its result is the exact top K over the index.
// Steps are enqueued back to back on one stream, two in flight, so the GPU
// never waits for the host's bookkeeping.
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
  int remaining = 0;  // rotating scan: queries of the request still in lanes
};

// Rotating scan: one step in flight (pinned host buffers are per step, reused
// only after the step's event has fired).
struct RotStep {
  cudaEvent_t done = nullptr;
  bool used = false;
  float *q_h = nullptr;                             // [max_q][dim] the step's queries
  int32_t *lane_h = nullptr, *k_h = nullptr;        // [max_q] batch row -> lane, K
  int32_t *reset_h = nullptr, *fin_h = nullptr;     // [max_q] lanes starting / finishing
  int32_t *ids_h = nullptr, *cnt_h = nullptr;       // [max_q][max_k], [max_q] finished rows
  float *sc_h = nullptr;
  std::vector<std::pair<Request *, int>> finished;  // (request, query) of each finished row
  lr_status status = LR_OK;
  std::string message;
};

struct RotLane {
  Request *r = nullptr;  // null: free
  int qi = 0;            // the request's query in this lane
  int steps = 0;         // chunks seen
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
  // rotating scan (chunks >= 2)
  int chunks = 1;
  int64_t chunk_rows = 0, n_rows = 0;
  Slot rot;  // its index context, stream and device query buffer
  int32_t *run_ids = nullptr, *run_cnt = nullptr, *c_ids = nullptr, *c_cnt = nullptr, *g_ids = nullptr,
          *g_cnt = nullptr, *lane_dev = nullptr, *k_dev = nullptr, *reset_dev = nullptr, *fin_dev = nullptr;
  float *run_sc = nullptr, *c_sc = nullptr, *g_sc = nullptr;
  RotStep ring[2];
  int ring_next = 0;
  std::vector<RotLane> lanes;
  std::vector<int32_t> new_lanes;  // admitted since the last step (reset before it merges)
  int64_t step = 0;
  int active = 0, terms_active = 0;
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

// ---------------------------------------------------------------- rotating scan

// Admit pending requests into free lanes, first come first served, while the
// whole request fits (lanes, term occurrences of the step's batch).  Lock held.
void rot_admit(lr_server *S) {
  const int cap = (int)S->lanes.size();
  while (!S->pending.empty()) {
    Request *r = S->pending.front();
    const int rt = (int)r->terms.size();
    if (S->active + r->B > cap || S->terms_active + rt > S->max_terms) break;
    S->pending.pop_front();
    r->remaining = r->B;
    r->ids.assign((size_t)r->B * r->k_max, -1);
    r->scores.assign((size_t)r->B * r->k_max, -INFINITY);
    r->count.assign(r->B, 0);
    int qi = 0;
    for (int l = 0; l < cap && qi < r->B; ++l) {
      if (S->lanes[l].r) continue;
      S->lanes[l] = RotLane{r, qi++, 0};
      S->new_lanes.push_back(l);
    }
    S->active += r->B;
    S->terms_active += rt;
  }
}

// Enqueue one step on the rotating stream: the chunk's search for every active
// lane, the merge into the lanes, and the rows of the lanes that have now seen
// every chunk copied to the step's pinned buffers.  Only the scheduler thread
// touches the lanes, so this runs without the lock.
void rot_launch(lr_server *S, RotStep &e) {
  const int cap = (int)S->lanes.size();
  const int c = (int)(S->step % S->chunks);
  const int64_t r0 = (int64_t)c * S->chunk_rows, r1 = std::min<int64_t>(S->n_rows, r0 + S->chunk_rows);
  std::vector<int32_t> q_off{0}, c_off{0}, k;
  std::vector<uint32_t> terms;
  int B = 0, k_all = 1, nf = 0;
  e.finished.clear();
  for (int l = 0; l < cap; ++l) {
    RotLane &ln = S->lanes[l];
    if (!ln.r) continue;
    Request *r = ln.r;
    std::memcpy(e.q_h + (size_t)B * S->dim, r->q.data() + (size_t)ln.qi * S->dim, sizeof(float) * S->dim);
    for (int cl = r->q_off[ln.qi]; cl < r->q_off[ln.qi + 1]; ++cl) {
      for (int t = r->c_off[cl]; t < r->c_off[cl + 1]; ++t) terms.push_back(r->terms[t]);
      c_off.push_back((int32_t)terms.size());
    }
    q_off.push_back((int32_t)c_off.size() - 1);
    k.push_back(r->k[ln.qi]);
    k_all = std::max(k_all, r->k[ln.qi]);
    e.lane_h[B] = l;
    e.k_h[B] = r->k[ln.qi];
    if (ln.steps + 1 == S->chunks) {
      e.fin_h[nf++] = l;
      e.finished.emplace_back(r, ln.qi);
    }
    ++B;
  }
  const int nr = (int)S->new_lanes.size();
  for (int i = 0; i < nr; ++i) e.reset_h[i] = S->new_lanes[i];
  S->new_lanes.clear();
  if (terms.empty()) terms.push_back(0);
  lr_filters f{q_off.data(), c_off.data(), terms.data()};
  lr_search_opts o = S->opts;
  o.row_begin = r0;
  o.row_end = r1;
  cudaStream_t st = S->rot.stream;
  lr_status status = LR_OK;
  auto ck = [&](cudaError_t err, const char *what) {
    if (err != cudaSuccess && status == LR_OK) status = fail(LR_ERR_CUDA, std::string("rotating scan: ") + what);
  };
  ck(cudaMemcpyAsync(S->rot.q_dev, e.q_h, sizeof(float) * (size_t)B * S->dim, cudaMemcpyHostToDevice, st), "upload");
  ck(cudaMemcpyAsync(S->lane_dev, e.lane_h, sizeof(int32_t) * B, cudaMemcpyHostToDevice, st), "upload");
  ck(cudaMemcpyAsync(S->k_dev, e.k_h, sizeof(int32_t) * B, cudaMemcpyHostToDevice, st), "upload");
  if (nr > 0) {
    ck(cudaMemcpyAsync(S->reset_dev, e.reset_h, sizeof(int32_t) * nr, cudaMemcpyHostToDevice, st), "upload");
    ck(launch_lane_reset(S->reset_dev, nr, S->run_cnt, st), "lane reset");
  }
  if (status == LR_OK)
    status = lr_search_ex(S->rot.ix, S->rot.q_dev, B, &f, k.data(), k_all, S->c_ids, S->c_sc, S->c_cnt, &o, nullptr,
                          st);
  if (status == LR_OK) {
    ck(launch_lane_merge(S->c_ids, S->c_sc, S->c_cnt, B, k_all, S->lane_dev, S->k_dev, S->run_ids, S->run_sc,
                         S->run_cnt, S->max_k, st),
       "lane merge");
    if (nf > 0) {
      const size_t rows = (size_t)nf * S->max_k;
      ck(cudaMemcpyAsync(S->fin_dev, e.fin_h, sizeof(int32_t) * nf, cudaMemcpyHostToDevice, st), "upload");
      ck(launch_lane_gather(S->fin_dev, nf, S->run_ids, S->run_sc, S->run_cnt, S->max_k, S->max_k, S->g_ids, S->g_sc,
                            S->g_cnt, st),
         "lane gather");
      ck(cudaMemcpyAsync(e.ids_h, S->g_ids, sizeof(int32_t) * rows, cudaMemcpyDeviceToHost, st), "download");
      ck(cudaMemcpyAsync(e.sc_h, S->g_sc, sizeof(float) * rows, cudaMemcpyDeviceToHost, st), "download");
      ck(cudaMemcpyAsync(e.cnt_h, S->g_cnt, sizeof(int32_t) * nf, cudaMemcpyDeviceToHost, st), "download");
    }
  }
  ck(cudaEventRecord(e.done, st), "event record");
  e.status = status;
  e.message = status == LR_OK ? std::string() : std::string(lr_last_error_message());
  // bookkeeping: every active lane saw this chunk; finished lanes are free for
  // the next step (their reset comes after this step's gather in stream order)
  for (int l = 0; l < cap; ++l) {
    RotLane &ln = S->lanes[l];
    if (!ln.r) continue;
    if (status != LR_OK && ln.r->status == LR_OK) {  // the request reports the step's failure
      ln.r->status = status;
      ln.r->message = e.message;
    }
    if (++ln.steps == S->chunks) ln = RotLane{};
  }
  S->active -= nf;
  e.used = true;
  ++S->step;
}

// Hand the rows of a finished step to their requests.  Lock held.
void rot_retire(lr_server *S, RotStep &e) {
  const Clock::time_point now = Clock::now();
  for (size_t j = 0; j < e.finished.size(); ++j) {
    Request *r = e.finished[j].first;
    const int qi = e.finished[j].second;
    if (e.status == LR_OK) {
      std::memcpy(&r->ids[(size_t)qi * r->k_max], e.ids_h + j * S->max_k, sizeof(int32_t) * r->k_max);
      std::memcpy(&r->scores[(size_t)qi * r->k_max], e.sc_h + j * S->max_k, sizeof(float) * r->k_max);
      r->count[qi] = std::min(e.cnt_h[j], r->k[qi]);
    } else if (r->status == LR_OK) {
      r->status = e.status;
      r->message = e.message;
    }
    if (--r->remaining == 0) {
      r->latency_ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
      r->done = true;
      S->lat.push_back(r->latency_ms);
      S->terms_active -= (int)r->terms.size();
      ++S->completed;
      S->queries += r->B;
    }
  }
  ++S->batches;
  e.finished.clear();
  e.used = false;
  S->cv_done.notify_all();
}

void rot_scheduler(lr_server *S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    bool inflight = false;
    for (RotStep &e : S->ring) {
      if (!e.used) continue;
      const cudaError_t err = cudaEventQuery(e.done);
      if (err == cudaSuccess) {
        rot_retire(S, e);
      } else {
        if (err == cudaErrorNotReady) cudaGetLastError();
        inflight = true;
      }
    }
    rot_admit(S);
    RotStep &e = S->ring[S->ring_next];
    if (S->active > 0 && !e.used) {
      lk.unlock();
      rot_launch(S, e);
      lk.lock();
      S->ring_next ^= 1;
      continue;
    }
    if (S->stop && S->pending.empty() && S->active == 0 && !inflight) break;
    if (inflight || S->active > 0) {
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

// The rotating scan's slot, lanes and per-step buffers (chunks >= 2).
lr_status rot_create(lr_server *S, lr_index *index, int chunks) {
  S->chunks = chunks;
  S->n_rows = index_rows(index);
  // chunk boundaries at multiples of 256 rows (the search's row-range rule)
  const int64_t groups = (S->n_rows + 255) / 256;
  S->chunk_rows = std::max<int64_t>(1, (groups + chunks - 1) / chunks) * 256;
  S->chunks = (int)((S->n_rows + S->chunk_rows - 1) / S->chunk_rows);  // no empty chunk
  lr_status st = index_clone_slot(index, S->max_q, nullptr, &S->rot.ix);
  if (st != LR_OK) return st;
  const size_t q = (size_t)S->max_q, rows = q * S->max_k;
  bool ok = cudaStreamCreateWithFlags(&S->rot.stream, cudaStreamNonBlocking) == cudaSuccess &&
            cudaMalloc(&S->rot.q_dev, sizeof(float) * q * S->dim) == cudaSuccess &&
            cudaMalloc(&S->run_ids, 4 * rows) == cudaSuccess && cudaMalloc(&S->run_sc, 4 * rows) == cudaSuccess &&
            cudaMalloc(&S->run_cnt, 4 * q) == cudaSuccess && cudaMalloc(&S->c_ids, 4 * rows) == cudaSuccess &&
            cudaMalloc(&S->c_sc, 4 * rows) == cudaSuccess && cudaMalloc(&S->c_cnt, 4 * q) == cudaSuccess &&
            cudaMalloc(&S->g_ids, 4 * rows) == cudaSuccess && cudaMalloc(&S->g_sc, 4 * rows) == cudaSuccess &&
            cudaMalloc(&S->g_cnt, 4 * q) == cudaSuccess && cudaMalloc(&S->lane_dev, 4 * q) == cudaSuccess &&
            cudaMalloc(&S->k_dev, 4 * q) == cudaSuccess && cudaMalloc(&S->reset_dev, 4 * q) == cudaSuccess &&
            cudaMalloc(&S->fin_dev, 4 * q) == cudaSuccess;
  for (RotStep &e : S->ring)
    ok = ok && cudaEventCreateWithFlags(&e.done, cudaEventDisableTiming) == cudaSuccess &&
         cudaHostAlloc((void **)&e.q_h, sizeof(float) * q * S->dim, 0) == cudaSuccess &&
         cudaHostAlloc((void **)&e.lane_h, 4 * q, 0) == cudaSuccess &&
         cudaHostAlloc((void **)&e.k_h, 4 * q, 0) == cudaSuccess &&
         cudaHostAlloc((void **)&e.reset_h, 4 * q, 0) == cudaSuccess &&
         cudaHostAlloc((void **)&e.fin_h, 4 * q, 0) == cudaSuccess &&
         cudaHostAlloc((void **)&e.ids_h, 4 * rows, 0) == cudaSuccess &&
         cudaHostAlloc((void **)&e.sc_h, 4 * rows, 0) == cudaSuccess &&
         cudaHostAlloc((void **)&e.cnt_h, 4 * q, 0) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return fail(LR_ERR_NOMEM, "cannot allocate the rotating scan's buffers");
  }
  S->max_terms = index_max_batch_terms(S->rot.ix);
  S->slot_bytes = lr_index_device_bytes(S->rot.ix) + sizeof(float) * q * S->dim + 32 * rows + 40 * q;
  S->lanes.assign(q, RotLane{});
  return LR_OK;
}

void rot_free(lr_server *S) {
  if (S->rot.stream) cudaStreamSynchronize(S->rot.stream);
  if (S->rot.ix) index_destroy_slot(S->rot.ix);
  for (void *p : {(void *)S->rot.q_dev, (void *)S->run_ids, (void *)S->run_sc, (void *)S->run_cnt, (void *)S->c_ids,
                  (void *)S->c_sc, (void *)S->c_cnt, (void *)S->g_ids, (void *)S->g_sc, (void *)S->g_cnt,
                  (void *)S->lane_dev, (void *)S->k_dev, (void *)S->reset_dev, (void *)S->fin_dev})
    cudaFree(p);
  for (RotStep &e : S->ring) {
    for (void *p : {(void *)e.q_h, (void *)e.lane_h, (void *)e.k_h, (void *)e.reset_h, (void *)e.fin_h, (void *)e.ids_h,
                    (void *)e.sc_h, (void *)e.cnt_h})
      cudaFreeHost(p);
    if (e.done) cudaEventDestroy(e.done);
  }
  if (S->rot.stream) cudaStreamDestroy(S->rot.stream);
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
  if (opts->chunks >= 2) {  // the rotating scan: one slot of max_queries lanes
    const lr_status st = rot_create(S, index, opts->chunks);
    if (st != LR_OK) {
      rot_free(S);
      delete S;
      return st;
    }
    S->t0 = Clock::now();
    S->th = std::thread(rot_scheduler, S);
    *out = S;
    return LR_OK;
  }
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
  st->slots = S->chunks >= 2 ? 1 : (int32_t)S->slots.size();
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
  if (S->chunks >= 2) rot_free(S);
  for (auto &kv : S->live) delete kv.second;
  delete S;
  return LR_OK;
}

}  // extern "C"
