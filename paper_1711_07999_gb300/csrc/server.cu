// server.cu -- continuous-batching frame server over tracking sessions (the serving calls of trk.h).
//
// A dispatcher thread keeps every attached session's frames flowing: a submitted frame is copied into a
// pinned staging buffer at once (buffers are pooled per session and reused once a frame is collected); as soon as its session has no frame on the GPU and one of the
// max_inflight slots is free, the frame is launched on the session's own stream (H2D of the depth, the
// session's frame graph, D2H of the results, an event).  Frames of different sessions therefore overlap
// on the device, new requests are admitted whenever a slot frees up, and one session's frames run in
// submission order (each starts from the state the previous one left).  Completion is detected by
// polling the events (no device-side waits); latency is wall time from submit to completion.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/trk.h"
#include "trk_internal.cuh"

namespace trk {
// defined in trk_api.cu
size_t session_device_bytes(const trk_session* s);
int session_device(const trk_session* s);
trk_status session_enqueue_frame(trk_session* s, const float* host_depth, cudaStream_t* stream_out);
trk_status session_enqueue_results(trk_session* s, double* theta, float* phi4, double* energy, int* stats);
void session_result_sizes(const trk_session* s, int* n_links, int* n_verts, int* n_energy);
}  // namespace trk

namespace {

using clk = std::chrono::steady_clock;

// Pinned staging of one frame of one session (reused: pinning host memory takes milliseconds).
struct Staging {
  float* depth = nullptr;     // pinned [H*W]
  double* theta = nullptr;    // pinned [L]
  float* phi4 = nullptr;      // pinned [V][4]
  double* energy = nullptr;   // pinned [pose + shape iters]
  int* stats = nullptr;       // pinned [4]
  cudaEvent_t done_ev = nullptr;
};

struct Request {
  uint64_t ticket = 0;
  trk_session* s = nullptr;
  Staging* b = nullptr;
  clk::time_point t_submit, t_done;
  int state = 0;              // 0 queued, 1 on the GPU, 2 done
  trk_status status = TRK_OK;
};

struct SessionSlot {
  std::deque<Request*> pending;
  Request* inflight = nullptr;
  std::vector<Staging*> spare;  // staging buffers of collected frames, ready for reuse
};

}  // namespace

struct trk_server {
  size_t budget = 0, used = 0;
  int max_inflight = 0, device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::map<trk_session*, SessionSlot> sessions;
  std::map<uint64_t, Request*> requests;
  uint64_t next_ticket = 1;
  int inflight = 0;
  bool stop = false;
  std::thread worker;
  std::vector<double> lat_us;  // completed frames
  uint64_t completed = 0;
};

namespace {

void free_staging(Staging* b) {
  if (!b) return;
  if (b->done_ev) cudaEventDestroy(b->done_ev);
  cudaFreeHost(b->depth);
  cudaFreeHost(b->theta);
  cudaFreeHost(b->phi4);
  cudaFreeHost(b->energy);
  cudaFreeHost(b->stats);
  delete b;
}

Staging* new_staging(size_t npx, int L, int V, int ne) {
  Staging* b = new Staging();
  const bool ok = cudaMallocHost(&b->depth, sizeof(float) * npx) == cudaSuccess &&
                  cudaMallocHost(&b->theta, sizeof(double) * L) == cudaSuccess &&
                  cudaMallocHost(&b->phi4, sizeof(float) * 4 * V) == cudaSuccess &&
                  cudaMallocHost(&b->energy, sizeof(double) * std::max(ne, 1)) == cudaSuccess &&
                  cudaMallocHost(&b->stats, sizeof(int) * 4) == cudaSuccess &&
                  cudaEventCreateWithFlags(&b->done_ev, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    free_staging(b);
    return nullptr;
  }
  return b;
}

void free_request(Request* r) {
  if (!r) return;
  free_staging(r->b);
  delete r;
}

// launches the next frame of every idle session while slots are free (lock held)
void launch_ready(trk_server* sv) {
  for (auto& kv : sv->sessions) {
    if (sv->inflight >= sv->max_inflight) return;
    SessionSlot& sl = kv.second;
    if (sl.inflight || sl.pending.empty()) continue;
    Request* r = sl.pending.front();
    sl.pending.pop_front();
    cudaStream_t st = nullptr;
    trk_status e = trk::session_enqueue_frame(r->s, r->b->depth, &st);
    if (e == TRK_OK) e = trk::session_enqueue_results(r->s, r->b->theta, r->b->phi4, r->b->energy, r->b->stats);
    if (e == TRK_OK && cudaEventRecord(r->b->done_ev, st) != cudaSuccess) e = TRK_ERR_CUDA;
    if (e != TRK_OK) {
      r->status = e;
      r->state = 2;
      r->t_done = clk::now();
      sv->cv_done.notify_all();
      continue;
    }
    r->state = 1;
    sl.inflight = r;
    ++sv->inflight;
  }
}

void worker_loop(trk_server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (!sv->stop) {
    launch_ready(sv);
    bool any = false;
    for (auto& kv : sv->sessions) {
      Request* r = kv.second.inflight;
      if (!r) continue;
      any = true;
      const cudaError_t q = cudaEventQuery(r->b->done_ev);
      if (q == cudaErrorNotReady) continue;
      r->status = q == cudaSuccess ? TRK_OK : TRK_ERR_CUDA;
      r->state = 2;
      r->t_done = clk::now();
      sv->lat_us.push_back(std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count());
      ++sv->completed;
      kv.second.inflight = nullptr;
      --sv->inflight;
      sv->cv_done.notify_all();
    }
    if (any) {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    } else {
      sv->cv_work.wait_for(lk, std::chrono::milliseconds(5));
    }
  }
}

}  // namespace

extern "C" {

trk_status trk_server_create(size_t hbm_budget_bytes, int32_t max_inflight, trk_server** out) {
  if (!out || max_inflight < 0) return trk::set_error(TRK_ERR_INVALID_ARG, "trk_server_create: bad arguments");
  trk_server* sv = new trk_server();
  sv->budget = hbm_budget_bytes;
  sv->max_inflight = max_inflight;
  cudaGetDevice(&sv->device);
  sv->worker = std::thread(worker_loop, sv);
  *out = sv;
  return TRK_OK;
}

trk_status trk_server_attach(trk_server* sv, trk_session* s) {
  if (!sv || !s) return trk::set_error(TRK_ERR_INVALID_ARG, "trk_server_attach: NULL argument");
  if (trk::session_device(s) != sv->device)
    return trk::set_error(TRK_ERR_INVALID_ARG, "trk_server_attach: session is on another device");
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->sessions.count(s)) return trk::set_error(TRK_ERR_INVALID_ARG, "trk_server_attach: already attached");
  const size_t need = trk::session_device_bytes(s);
  if (sv->used + need > sv->budget)
    return trk::set_error(TRK_ERR_NO_CAPACITY, "trk_server_attach: the session does not fit the HBM budget");
  sv->used += need;
  sv->sessions[s];
  return TRK_OK;
}

trk_status trk_server_detach(trk_server* sv, trk_session* s) {
  if (!sv || !s) return trk::set_error(TRK_ERR_INVALID_ARG, "trk_server_detach: NULL argument");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->sessions.find(s);
  if (it == sv->sessions.end()) return trk::set_error(TRK_ERR_INVALID_ARG, "trk_server_detach: not attached");
  if (!it->second.pending.empty() || it->second.inflight)
    return trk::set_error(TRK_ERR_INVALID_ARG, "trk_server_detach: the session still has frames");
  sv->used -= trk::session_device_bytes(s);
  for (Staging* b : it->second.spare) free_staging(b);
  sv->sessions.erase(it);
  return TRK_OK;
}

trk_status trk_server_submit(trk_server* sv, trk_session* s, const float* depth_m, uint64_t* ticket) {
  if (!sv || !s || !depth_m || !ticket) return trk::set_error(TRK_ERR_INVALID_ARG, "trk_server_submit: NULL argument");
  int L = 0, V = 0, ne = 0;
  trk::session_result_sizes(s, &L, &V, &ne);
  trk_info inf;
  trk_get_info(s, &inf);
  const size_t npx = (size_t)inf.width * inf.height;
  Request* r = new Request();
  r->s = s;
  r->t_submit = clk::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->sessions.find(s);
    if (it == sv->sessions.end()) {
      delete r;
      return trk::set_error(TRK_ERR_INVALID_ARG, "trk_server_submit: session not attached");
    }
    if (!it->second.spare.empty()) {
      r->b = it->second.spare.back();
      it->second.spare.pop_back();
    }
  }
  if (!r->b && !(r->b = new_staging(npx, L, V, ne))) {
    delete r;
    return trk::set_error(TRK_ERR_OOM, "trk_server_submit: pinned staging allocation failed");
  }
  std::memcpy(r->b->depth, depth_m, sizeof(float) * npx);
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->sessions.find(s);
    if (it == sv->sessions.end()) {  // detached meanwhile
      free_request(r);
      return trk::set_error(TRK_ERR_INVALID_ARG, "trk_server_submit: session not attached");
    }
    r->ticket = sv->next_ticket++;
    sv->requests[r->ticket] = r;
    it->second.pending.push_back(r);
    *ticket = r->ticket;
  }
  sv->cv_work.notify_one();
  return TRK_OK;
}

trk_status trk_server_wait(trk_server* sv, uint64_t ticket, int64_t timeout_us, trk_result* out) {
  if (!sv) return trk::set_error(TRK_ERR_INVALID_ARG, "trk_server_wait: NULL server");
  std::unique_lock<std::mutex> lk(sv->mu);
  const auto deadline = clk::now() + std::chrono::microseconds(std::max<int64_t>(timeout_us, 0));
  Request* r = nullptr;
  for (;;) {  // look the ticket up again after every wake-up: another waiter may have taken it
    auto it = sv->requests.find(ticket);
    if (it == sv->requests.end()) return trk::set_error(TRK_ERR_INVALID_ARG, "trk_server_wait: unknown ticket");
    if (it->second->state == 2) {
      r = it->second;
      sv->requests.erase(it);
      break;
    }
    if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
      auto again = sv->requests.find(ticket);
      if (again == sv->requests.end() || again->second->state != 2)
        return trk::set_error(TRK_ERR_TIMEOUT, "trk_server_wait: the frame is not done yet");
    }
  }
  lk.unlock();
  const Staging* b = r->b;
  trk_status st = r->status;
  if (st == TRK_OK && b->stats[3]) st = trk::set_error(TRK_ERR_TIMEOUT, "trk_server_wait: a tensor-core wait ran out");
  if (st == TRK_OK && out) {
    int L = 0, V = 0, ne = 0;
    trk::session_result_sizes(r->s, &L, &V, &ne);
    if (out->theta) std::memcpy(out->theta, b->theta, sizeof(double) * L);
    if (out->energy) std::memcpy(out->energy, b->energy, sizeof(double) * ne);
    if (out->offsets)
      for (int i = 0; i < V; ++i)
        for (int c = 0; c < 3; ++c) out->offsets[3 * i + c] = b->phi4[4 * i + c];
    out->n_assoc_px = b->stats[0];
    out->n_assoc_verts = b->stats[1];
  }
  lk.lock();  // the staging goes back to its session (or is freed if the session left meanwhile)
  auto it = sv->sessions.find(r->s);
  if (it != sv->sessions.end()) {
    it->second.spare.push_back(r->b);
    r->b = nullptr;
  }
  lk.unlock();
  free_request(r);
  if (st != TRK_OK) return trk::set_error(st, "trk_server_wait: the frame failed on the device");
  return TRK_OK;
}

trk_status trk_server_get_stats(trk_server* sv, trk_server_stats* out) {
  if (!sv || !out) return trk::set_error(TRK_ERR_INVALID_ARG, "trk_server_get_stats: NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  out->frames_done = sv->completed;
  out->in_flight = sv->inflight;
  out->sessions = (int32_t)sv->sessions.size();
  out->hbm_used_bytes = sv->used;
  std::vector<double> l = sv->lat_us;
  out->latency_p50_us = out->latency_p99_us = out->latency_max_us = 0.0;
  if (!l.empty()) {
    std::sort(l.begin(), l.end());
    auto pct = [&](double p) { return l[std::min(l.size() - 1, (size_t)(p * (l.size() - 1) + 0.5))]; };
    out->latency_p50_us = pct(0.50);
    out->latency_p99_us = pct(0.99);
    out->latency_max_us = l.back();
  }
  return TRK_OK;
}

void trk_server_destroy(trk_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  for (auto& kv : sv->sessions) {
    if (kv.second.inflight) cudaEventSynchronize(kv.second.inflight->b->done_ev);
    for (Staging* b : kv.second.spare) free_staging(b);
  }
  for (auto& kv : sv->requests) free_request(kv.second);
  delete sv;
}

}  // extern "C"
