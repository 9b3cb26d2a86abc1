// The request server: continuous batching of MAPE instances on one GPU.
//
// Requests (an instance, its starts and its augmentation starts) are copied
// at submission and queued.  A scheduler thread admits them in arrival order
// while a slot is free and the device-memory estimate of the running requests
// plus the next one stays within the cap; an admitted request runs on its
// slot's own stream through an instance handle (extraction, filtering, then
// Algorithm 1 from its starts), so the work of all running requests overlaps
// on the device, and a request that arrives while others run is admitted as
// soon as a slot and memory free up.  Each request records, on the server's
// clock, its submission, admission, end of extraction, first improving move
// and completion; its results (best x, f, and optionally the direction set)
// stay on the host after its device memory is released.
#include "common.cuh"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

namespace {

double clock_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t id = 0;
  int n = 0, m = 0, P = 0, S = 0;
  std::vector<int32_t> A, l, u, Q, c, w, B, X0;
  std::vector<int64_t> b;
  std::vector<float> Z0, G0;
  bool has_w = false;
  size_t bytes = 0;
  // progress
  int state = MAPE_REQ_QUEUED;
  int error = MAPE_OK;
  int stage = 0;  // 1: extracting, 2: augmenting, 3: waiting for an augmentation batch
  mape_handle h = nullptr;
  int slot = -1;
  bool ready = false;  // batch mode: handle created, extraction not started yet
  double t_ready = 0;
  bool aug_ready = false;  // batch mode: directions found, augmentation not started yet
  double t_aug_ready = 0;
  double t_submit = 0, t_admit = 0, t_extracted = 0, t_first = 0, t_done = 0;
  // results
  int64_t directions = 0, best_f = 0, aug_iters = 0;
  std::vector<int32_t> x;
  std::vector<int8_t> G;  // K x n, when kept
};

}  // namespace

struct mape_server {
  mape_server_config cfg{};
  int dev = 0;
  std::vector<cudaStream_t> streams;
  std::vector<bool> slot_busy;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<uint64_t> queue;
  std::map<uint64_t, std::unique_ptr<Request>> reqs;
  uint64_t next_id = 1;
  size_t mem_in_use = 0, mem_peak = 0;
  int running = 0, peak_running = 0;
  int64_t submitted = 0, completed = 0, failed = 0;
  bool stop = false;
  std::thread sched;
  int starting = 0;  // admitted requests whose handle is being created (under mu)

  void loop();
  void start(Request* r, int slot);
  void start_batch(std::vector<Request*>& rs);
  void advance(Request* r);
  void finish(Request* r, int err);
};

// Device bytes a request holds while it runs: what mape_create_instance,
// mape_extract_directions and mape_augment allocate for these sizes.
extern "C" size_t mape_request_bytes(int32_t n, int32_t m, int32_t P, int32_t S, const mape_config* cfg) {
  if (n <= 0 || m <= 0 || m >= n || P <= 0 || S <= 0 || !cfg) return 0;
  using mape_detail::align_up;
  const size_t d = (size_t)(n - m), N = (size_t)n, ldg = align_up(N, 16);
  const int64_t T = cfg->T > 0 ? cfg->T : 1;
  const int64_t period = cfg->period > 0 ? cfg->period : 1;
  int64_t cap = cfg->cand_capacity > 0 ? cfg->cand_capacity
                                       : mape_detail::default_cand_capacity(P, T / period, (int64_t)ldg);
  cap = std::max<int64_t>(cap, (int64_t)P + 1);
  size_t inst = (size_t)m * N * 4 + N * d * 4 + (size_t)m * 8 + 3 * N * 4 + 4;  // A, B, b, l, u, span
  inst += N * N * 12 / 8 + 2 * N * 4;                                            // Q as COO (bound), c, w
  inst += N * d * 4 + mape_project_prepare_workspace_bytes(n, (int32_t)d);      // W and its workspace
  size_t job = 3 * (size_t)P * d * 4 + (size_t)P * N * 4;                        // Z, M, V, G0
  job += 2 * (size_t)cap * ldg + 2 * (size_t)cap + 2 * (size_t)cap * 8 + 16;     // candidate buffers, flags, a, q4
  size_t w = mape_extract_workspace_bytes(n, (int32_t)d, P, cfg->precision);
  w = std::max(w, mape_dedup_workspace_bytes(cap, (int32_t)ldg));
  w = std::max(w, mape_kernel_test_workspace_bytes(m, n));
  w = std::max(w, mape_minimal_workspace_bytes(cap, n));
  job += w;
  size_t aug = (size_t)S * N * 4 + (size_t)S * 8 + 4;
  // the augmentation workspace grows with the direction count, bounded by cap
  aug += mape_augment_workspace_bytes(n, S, cap);
  return inst + job + aug + (64u << 10);  // allocation rounding
}

extern "C" int mape_server_create(const mape_server_config* sc, mape_server_h* out) {
  if (!out || !sc) return MAPE_ERR_INVALID_ARG;
  *out = nullptr;
  if (sc->max_slots <= 0 || sc->max_slots > 256 || sc->mem_cap_bytes == 0) return MAPE_ERR_INVALID_ARG;
  if (sc->batch_extraction) {
    const int32_t base = sc->cfg.precision & MAPE_PREC_MASK;
    if ((base != MAPE_PREC_BF16 && base != MAPE_PREC_BF16X1) || (sc->cfg.precision & MAPE_PREC_SPARSE_FWD))
      return MAPE_ERR_INVALID_ARG;
  }
  auto* s = new mape_server();
  s->cfg = *sc;
  if (cudaGetDevice(&s->dev) != cudaSuccess) {
    delete s;
    return MAPE_ERR_CUDA;
  }
  for (int i = 0; i < sc->max_slots; ++i) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto x : s->streams) cudaStreamDestroy(x);
      delete s;
      return MAPE_ERR_CUDA;
    }
    s->streams.push_back(st);
  }
  s->slot_busy.assign(sc->max_slots, false);
  s->sched = std::thread([s]() {
    cudaSetDevice(s->dev);
    s->loop();
  });
  *out = s;
  return MAPE_OK;
}

extern "C" int mape_server_submit(mape_server_h s, const int32_t* A, const int64_t* b, const int32_t* l,
                                  const int32_t* u, const mape_problem* f, const int32_t* B, int32_t P,
                                  const float* Z0, const float* G0, const int32_t* X0, int32_t S, uint64_t* id) {
  if (!s || !A || !b || !l || !u || !f || !f->Q || !f->c || !B || !X0 || !id || P <= 0 || S <= 0)
    return MAPE_ERR_INVALID_ARG;
  if ((Z0 == nullptr) == (G0 == nullptr)) return MAPE_ERR_INVALID_ARG;
  const int n = f->n, m = f->m;
  if (n <= 0 || m <= 0 || m >= n || n > 4096) return MAPE_ERR_SHAPE;
  const size_t bytes = mape_request_bytes(n, m, P, S, &s->cfg.cfg);
  if (bytes == 0) return MAPE_ERR_INVALID_ARG;
  if (bytes > s->cfg.mem_cap_bytes) return MAPE_ERR_OOM;  // could never be admitted
  auto r = std::make_unique<Request>();
  const int d = n - m;
  r->n = n; r->m = m; r->P = P; r->S = S; r->bytes = bytes;
  r->A.assign(A, A + (size_t)m * n);
  r->b.assign(b, b + m);
  r->l.assign(l, l + n);
  r->u.assign(u, u + n);
  r->Q.assign(f->Q, f->Q + (size_t)n * n);
  r->c.assign(f->c, f->c + n);
  r->has_w = f->w != nullptr;
  if (f->w) r->w.assign(f->w, f->w + n);
  r->B.assign(B, B + (size_t)n * d);
  if (Z0) r->Z0.assign(Z0, Z0 + (size_t)P * d);
  if (G0) r->G0.assign(G0, G0 + (size_t)P * n);
  r->X0.assign(X0, X0 + (size_t)S * n);
  std::lock_guard<std::mutex> lk(s->mu);
  r->id = s->next_id++;
  r->t_submit = clock_ms();
  *id = r->id;
  s->queue.push_back(r->id);
  s->reqs[r->id] = std::move(r);
  ++s->submitted;
  s->cv.notify_all();
  return MAPE_OK;
}

// Creates the handle on the slot's stream and starts its extraction.  Runs on
// a thread of its own per admission, without the lock (the uploads, the basis
// check and the projection's factorisation synchronise the slot's stream
// only), so that the scheduler keeps admitting and advancing requests while
// the handles of several admissions are being set up.
void mape_server::start(Request* r, int slot) {
  mape_problem f{r->n, r->m, r->Q.data(), r->c.data(), r->has_w ? r->w.data() : nullptr};
  mape_handle h = nullptr;
  int rc = mape_create_instance(r->A.data(), r->b.data(), r->l.data(), r->u.data(), &f, r->B.data(), &cfg.cfg,
                                streams[slot], &h);
  if (rc == MAPE_OK && !cfg.batch_extraction)
    rc = mape_extract_directions(h, r->P, r->Z0.empty() ? nullptr : r->Z0.data(),
                                 r->G0.empty() ? nullptr : r->G0.data());
  std::lock_guard<std::mutex> lk(mu);
  r->h = h;
  --starting;
  if (rc != MAPE_OK) {
    finish(r, rc);
    return;
  }
  if (cfg.batch_extraction) {  // the scheduler starts its extraction with the next batch
    r->ready = true;
    r->t_ready = clock_ms();
  } else {
    r->stage = 1;
  }
  cv.notify_all();
}

// Batch mode: the extraction of every request whose handle is ready runs as
// one mape_extract_directions_batch call (one graph of persistent launches
// per chunk of steps for all of them).  Called without the lock.
void mape_server::start_batch(std::vector<Request*>& rs) {
  std::vector<mape_handle> hs;
  std::vector<int32_t> P;
  std::vector<const float*> Z0, G0;
  for (auto r : rs) {
    hs.push_back(r->h);
    P.push_back(r->P);
    Z0.push_back(r->Z0.empty() ? nullptr : r->Z0.data());
    G0.push_back(r->G0.empty() ? nullptr : r->G0.data());
  }
  const int rc = mape_extract_directions_batch(hs.data(), (int32_t)hs.size(), P.data(), Z0.data(), G0.data());
  std::lock_guard<std::mutex> lk(mu);
  for (auto r : rs) {
    if (rc != MAPE_OK) finish(r, rc);
    else r->stage = 1;
  }
  --starting;
  cv.notify_all();
}

// Called with the lock held: releases the request's slot and memory.
void mape_server::finish(Request* r, int err) {
  if (r->h) {
    mape_destroy(r->h);
    r->h = nullptr;
  }
  r->error = err;
  r->state = err == MAPE_OK ? MAPE_REQ_DONE : MAPE_REQ_FAILED;
  r->t_done = clock_ms();
  if (err == MAPE_OK) ++completed; else ++failed;
  if (r->slot >= 0) slot_busy[r->slot] = false;
  r->slot = -1;
  mem_in_use -= r->bytes;
  --running;
  // the staged inputs are no longer needed
  std::vector<int32_t>().swap(r->A); std::vector<int32_t>().swap(r->B); std::vector<int32_t>().swap(r->Q);
  std::vector<float>().swap(r->Z0); std::vector<float>().swap(r->G0);
  cv.notify_all();
}

// Moves a running request on when its handle has finished a job.  Called with
// the lock held; the calls it makes do not block on other requests.
void mape_server::advance(Request* r) {
  if (r->stage == 3) return;  // the scheduler starts its augmentation with the next batch
  mape_status st{};
  mape_poll(r->h, &st);
  if (st.phase == MAPE_PHASE_ERROR) {
    finish(r, st.error ? st.error : MAPE_ERR_CUDA);
    return;
  }
  if (st.phase != MAPE_PHASE_DONE) return;
  if (r->stage == 1) {
    r->t_extracted = clock_ms();
    r->directions = st.directions;
    if (cfg.keep_directions && st.directions > 0) {
      std::vector<int32_t> G((size_t)st.directions * r->n);
      int64_t K = 0;
      int rc = mape_get_directions(r->h, G.data(), st.directions, &K);
      if (rc != MAPE_OK) { finish(r, rc); return; }
      r->G.resize(G.size());
      for (size_t i = 0; i < G.size(); ++i) r->G[i] = (int8_t)G[i];
    }
    if (cfg.batch_extraction) {
      r->aug_ready = true;
      r->t_aug_ready = clock_ms();
      r->stage = 3;
      return;
    }
    int rc = mape_augment(r->h, r->X0.data(), r->S, nullptr);
    if (rc != MAPE_OK) { finish(r, rc); return; }
    r->stage = 2;
    return;
  }
  // augmentation finished
  r->t_first = r->t_extracted + st.first_improve_ms;
  r->best_f = st.best_f;
  r->aug_iters = st.aug_iters;
  r->x.resize(r->n);
  int64_t fx = 0;
  int rc = mape_get_solution(r->h, r->x.data(), &fx);
  finish(r, rc);
}

void mape_server::loop() {
  std::unique_lock<std::mutex> lk(mu);
  while (!stop) {
    for (auto& kv : reqs) {
      Request* r = kv.second.get();
      if (r->state == MAPE_REQ_RUNNING && r->h && r->stage > 0) advance(r);
    }
    // batch mode: the requests whose handles are ready start their extraction
    // together, once no admitted request is still being set up or the oldest
    // ready one has waited 5 ms
    if (cfg.batch_extraction) {
      std::vector<Request*> ready;
      double oldest = 1e300;
      for (auto& kv : reqs) {
        Request* r = kv.second.get();
        if (r->state == MAPE_REQ_RUNNING && r->ready) {
          ready.push_back(r);
          oldest = std::min(oldest, r->t_ready);
        }
      }
      if (!ready.empty() && (starting == 0 || clock_ms() - oldest > 5.0)) {
        for (auto r : ready) r->ready = false;
        ++starting;  // the batch's uploads run on a thread of their own, like a request's set-up
        std::thread([this, ready]() mutable {
          cudaSetDevice(dev);
          start_batch(ready);
        }).detach();
      }
      // ... and the requests whose directions are found start Algorithm 1
      // together (mape_augment_batch), once no request is still extracting or
      // the oldest waiting one has waited 5 ms
      std::vector<Request*> aug;
      double aug_oldest = 1e300;
      bool extracting = false;
      for (auto& kv : reqs) {
        Request* r = kv.second.get();
        if (r->state != MAPE_REQ_RUNNING) continue;
        if (r->stage == 1 || r->ready) extracting = true;
        if (r->aug_ready) {
          aug.push_back(r);
          aug_oldest = std::min(aug_oldest, r->t_aug_ready);
        }
      }
      if (!aug.empty() && (!extracting || clock_ms() - aug_oldest > 5.0)) {
        // the starts' uploads and feasibility checks run on a thread of their
        // own (the requests stay at stage 3, which advance() skips, until the
        // batch has started)
        for (auto r : aug) r->aug_ready = false;
        ++starting;
        std::thread([this, aug]() {
          cudaSetDevice(dev);
          std::vector<mape_handle> hs;
          std::vector<const int32_t*> X0;
          std::vector<int32_t> S;
          for (auto r : aug) {
            hs.push_back(r->h);
            X0.push_back(r->X0.data());
            S.push_back(r->S);
          }
          const int rc = mape_augment_batch(hs.data(), (int32_t)hs.size(), X0.data(), S.data());
          std::lock_guard<std::mutex> lk(mu);
          for (auto r : aug) {
            if (rc != MAPE_OK) finish(r, rc);
            else r->stage = 2;
          }
          --starting;
          cv.notify_all();
        }).detach();
      }
    }
    // admission, in arrival order, while a slot and the memory allow
    while (!queue.empty()) {
      Request* r = reqs[queue.front()].get();
      int slot = -1;
      for (int i = 0; i < (int)slot_busy.size(); ++i)
        if (!slot_busy[i]) { slot = i; break; }
      if (slot < 0 || mem_in_use + r->bytes > cfg.mem_cap_bytes) break;
      queue.pop_front();
      slot_busy[slot] = true;
      r->slot = slot;
      r->state = MAPE_REQ_RUNNING;
      r->t_admit = clock_ms();
      mem_in_use += r->bytes;
      mem_peak = std::max(mem_peak, mem_in_use);
      ++running;
      peak_running = std::max(peak_running, running);
      ++starting;
      std::thread([this, r, slot] {
        cudaSetDevice(dev);
        start(r, slot);
      }).detach();
    }
    cv.wait_for(lk, std::chrono::microseconds(200));
  }
}

extern "C" int mape_server_poll(mape_server_h s, uint64_t id, mape_request_info* info) {
  if (!s || !info) return MAPE_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return MAPE_ERR_INVALID_ARG;
  const Request* r = it->second.get();
  std::memset(info, 0, sizeof(*info));
  info->state = r->state;
  info->error = r->error;
  info->n = r->n;
  info->m = r->m;
  info->P = r->P;
  info->directions = r->directions;
  info->best_f = r->best_f;
  info->aug_iters = r->aug_iters;
  info->bytes = r->bytes;
  info->t_submit_ms = r->t_submit;
  info->t_admit_ms = r->t_admit;
  info->t_extracted_ms = r->t_extracted;
  info->t_first_improve_ms = r->t_first;
  info->t_done_ms = r->t_done;
  return MAPE_OK;
}

extern "C" int mape_server_wait(mape_server_h s, uint64_t id, int64_t timeout_ns) {
  if (!s) return MAPE_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return MAPE_ERR_INVALID_ARG;
  Request* r = it->second.get();
  bool done = s->cv.wait_for(lk, std::chrono::nanoseconds(timeout_ns < 0 ? 0 : timeout_ns), [r] {
    return r->state == MAPE_REQ_DONE || r->state == MAPE_REQ_FAILED;
  });
  if (!done) return MAPE_ERR_TIMEOUT;
  return r->error;
}

extern "C" int mape_server_wait_all(mape_server_h s, int64_t timeout_ns) {
  if (!s) return MAPE_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  bool done = s->cv.wait_for(lk, std::chrono::nanoseconds(timeout_ns < 0 ? 0 : timeout_ns),
                             [s] { return s->queue.empty() && s->running == 0; });
  return done ? MAPE_OK : MAPE_ERR_TIMEOUT;
}

extern "C" int mape_server_result(mape_server_h s, uint64_t id, int32_t* x, int64_t* fval, int8_t* G, int64_t cap,
                                  int64_t* K) {
  if (!s) return MAPE_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return MAPE_ERR_INVALID_ARG;
  const Request* r = it->second.get();
  if (r->state != MAPE_REQ_DONE) return r->state == MAPE_REQ_FAILED ? r->error : MAPE_ERR_STATE;
  if (x) std::memcpy(x, r->x.data(), sizeof(int32_t) * r->n);
  if (fval) *fval = r->best_f;
  if (K) {
    const int64_t rows = r->n > 0 ? (int64_t)(r->G.size() / r->n) : 0;
    *K = rows;
    if (G) {
      if (cap < rows) return MAPE_ERR_CAPACITY;
      std::memcpy(G, r->G.data(), r->G.size());
    }
  }
  return MAPE_OK;
}

extern "C" int mape_server_release(mape_server_h s, uint64_t id) {
  if (!s) return MAPE_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return MAPE_ERR_INVALID_ARG;
  if (it->second->state != MAPE_REQ_DONE && it->second->state != MAPE_REQ_FAILED) return MAPE_ERR_STATE;
  s->reqs.erase(it);
  return MAPE_OK;
}

extern "C" int mape_server_get_stats(mape_server_h s, mape_server_stats* st) {
  if (!s || !st) return MAPE_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(st, 0, sizeof(*st));
  st->submitted = s->submitted;
  st->completed = s->completed;
  st->failed = s->failed;
  st->queued = (int64_t)s->queue.size();
  st->running = s->running;
  st->peak_running = s->peak_running;
  st->mem_in_use = s->mem_in_use;
  st->mem_peak = s->mem_peak;
  st->mem_cap = s->cfg.mem_cap_bytes;
  return MAPE_OK;
}

extern "C" void mape_server_destroy(mape_server_h s) {
  if (!s) return;
  mape_server_wait_all(s, (int64_t)600 * 1000000000ll);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  if (s->sched.joinable()) s->sched.join();
  {  // the threads that set up admitted requests finish on their own (bounded)
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv.wait_for(lk, std::chrono::seconds(600), [s] { return s->starting == 0; });
  }
  for (auto& kv : s->reqs)
    if (kv.second->h) {
      mape_cancel(kv.second->h);
      mape_wait(kv.second->h, (int64_t)60 * 1000000000ll);
      mape_destroy(kv.second->h);
    }
  for (auto st : s->streams) cudaStreamDestroy(st);
  delete s;
}
