// server.cu -- continuous-batching frame server over tracking sessions (the serving calls of trk.h).
//
// Sessions are admitted under an HBM budget: an evicted session (no device memory) gets its device state
// at trk_server_attach and gives it back at trk_server_detach, so the budget bounds what the server's
// sessions hold on the device.  A submitted frame is copied at once into host-mapped pinned staging and
// queued on its session.  A dispatcher thread launches frames as soon as their session has no frame on
// the GPU:
//  - batched dispatch (default): the ready frames of compatible sessions (same iteration schedule,
//    precision, association and tracking mode) go into ONE batched frame -- every stage one launch over
//    the blocks of all of them (trk::batch_step_launch) -- on one of a few step streams; the kernels
//    read the depth straight from the staging and write the results straight into it;
//  - per-session dispatch: each frame runs its session's own frame graph on the session's stream.
// Either way frames of different sessions overlap on the device, requests that arrive while others run
// are launched as soon as a step slot frees, and one session's frames run in submission order (each
// starts from the state the previous one left).  Completion comes from a host function enqueued behind
// each step (no polling); latency is wall time from submit to that point, kept in a fixed log-spaced
// histogram.
#include <algorithm>
#include <chrono>
#include <cmath>
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
bool session_resident(const trk_session* s);
trk_status session_evict(trk_session* s);
trk_status session_restore(trk_session* s);
const trk_params& session_params(const trk_session* s);
trk_status session_enqueue_frame(trk_session* s, const float* host_depth, cudaStream_t* stream_out);
trk_status session_enqueue_results(trk_session* s, double* theta, float* phi4, double* energy, int* stats);
void session_result_sizes(const trk_session* s, int* n_links, int* n_verts, int* n_energy);
void session_forget_stream(trk_session* s, cudaStream_t st);
}  // namespace trk

namespace {

using clk = std::chrono::steady_clock;

// Submit-to-completion latencies: log-spaced bins from 1 us to 1e8 us, 200 per decade (each bin 1.16 %
// wide), plus the exact maximum.  Fixed size however long the server runs.
struct LatencyHistogram {
  static constexpr int kPerDecade = 200, kDecades = 8, kBins = kPerDecade * kDecades + 2;
  uint64_t bins[kBins] = {};
  uint64_t n = 0;
  double max_us = 0.0;
  static int bin_of(double us) {
    if (!(us >= 1.0)) return 0;
    const int b = 1 + (int)std::floor(std::log10(us) * kPerDecade);
    return std::min(b, kBins - 1);
  }
  static double upper_edge(int b) { return b == 0 ? 1.0 : std::pow(10.0, (double)b / kPerDecade); }
  void add(double us) {
    ++bins[bin_of(us)];
    ++n;
    max_us = std::max(max_us, us);
  }
  // the upper edge of the first bin at which the cumulative count reaches p n (capped by the maximum)
  double percentile(double p) const {
    if (!n) return 0.0;
    const double want = std::max(1.0, std::ceil(p * (double)n));
    uint64_t c = 0;
    for (int b = 0; b < kBins; ++b) {
      c += bins[b];
      if ((double)c >= want) return std::min(upper_edge(b), max_us);
    }
    return max_us;
  }
};

// Pinned, host-mapped staging of one frame: the depth the kernels read and the results they write.
struct Staging {
  void* block = nullptr;  // one cudaHostAlloc'd block
  size_t npx = 0;
  int L = 0, V = 0, ne = 0;  // capacity
  float* depth = nullptr;    // [npx]
  double* theta = nullptr;   // [L]
  double* energy = nullptr;  // [ne]
  int* stats = nullptr;      // [4]
  float4* phi = nullptr;     // [V]
  const float* depth_dev = nullptr;  // device addresses of the same memory
  trk::ResultDst dst{};
};

struct Request;
struct Step {
  trk_server* sv = nullptr;
  cudaStream_t st = nullptr;       // a batched slot's own stream, or the session's stream
  trk::BatchStep* bs = nullptr;    // buffers of a batched slot (nullptr: one session's frame graph)
  std::vector<Request*> reqs;
  clk::time_point t_done;
  bool busy = false;
};

struct Request {
  uint64_t ticket = 0;
  trk_session* s = nullptr;
  Staging* b = nullptr;
  clk::time_point t_submit, t_done;
  int state = 0;  // 0 queued, 1 on the GPU, 2 done
  trk_status status = TRK_OK;
};

struct SessionSlot {
  std::deque<Request*> pending;
  Request* inflight = nullptr;
  std::vector<Staging*> spare;  // staging of collected frames, ready for reuse
  size_t bytes = 0;             // the session's arena, counted against the budget
  size_t step_bytes = 0;        // its tables in a batched step
  bool restored = false;        // made resident at attach (evicted again at detach)
  bool batchable = false;       // tracking mode: may join batched steps
  uint64_t key = 0;             // sessions with equal keys may share a batched step
};

}  // namespace

struct trk_server {
  size_t budget = 0, used = 0;      // used: arena_used + the step buffers' reservation
  size_t arena_used = 0;            // the arenas of the attached (and attaching) sessions
  size_t step_sum = 0, step_peak = 0;  // their step-table bytes now, and the most there have been
  size_t gran = 2 << 20;            // the device's allocation granularity
  int max_inflight = 0, device = 0;
  int dispatch = TRK_SERVER_DISPATCH_BATCHED;
  int max_batch = 64, n_slots = 2;
  int64_t max_wait_us = 2000;       // longest a ready frame waits for a fuller step while another runs
  clk::time_point wake{};           // when the dispatcher must look again (a waiting frame's deadline)
  bool wake_set = false;
  std::mutex mu;                    // sessions, requests, counters (held while launching)
  std::condition_variable cv_done;  // a frame completed
  std::mutex sig_mu;                // finished steps and the work flag (never held across a CUDA call)
  std::condition_variable cv_sig;
  std::vector<Step*> finished;
  bool work = false, stop = false;
  std::map<trk_session*, SessionSlot> sessions;
  std::map<trk_session*, bool> attaching;
  std::map<uint64_t, Request*> requests;
  std::vector<Step*> slots;         // batched step slots
  std::vector<Staging*> pool;       // staging given back by departed sessions
  uint64_t next_ticket = 1;
  int inflight = 0;
  std::thread worker;
  LatencyHistogram lat;
  uint64_t completed = 0, steps = 0, frames_in_steps = 0;
};

namespace {

void free_staging(Staging* b) {
  if (!b) return;
  cudaFreeHost(b->block);
  delete b;
}

size_t up16(size_t x) { return (x + 15) & ~size_t(15); }

Staging* new_staging(size_t npx, int L, int V, int ne) {
  Staging* b = new Staging();
  const size_t o_th = up16(sizeof(float) * npx), o_en = o_th + up16(sizeof(double) * L),
               o_st = o_en + up16(sizeof(double) * std::max(ne, 1)), o_phi = o_st + 16,
               total = o_phi + sizeof(float4) * std::max(V, 1);
  if (cudaHostAlloc(&b->block, total, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
    delete b;
    return nullptr;
  }
  char* dev = nullptr;
  if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&dev), b->block, 0) != cudaSuccess) {
    free_staging(b);
    return nullptr;
  }
  char* h = static_cast<char*>(b->block);
  b->npx = npx;
  b->L = L;
  b->V = V;
  b->ne = ne;
  b->depth = reinterpret_cast<float*>(h);
  b->theta = reinterpret_cast<double*>(h + o_th);
  b->energy = reinterpret_cast<double*>(h + o_en);
  b->stats = reinterpret_cast<int*>(h + o_st);
  b->phi = reinterpret_cast<float4*>(h + o_phi);
  b->depth_dev = reinterpret_cast<const float*>(dev);
  b->dst.theta = reinterpret_cast<double*>(dev + o_th);
  b->dst.energy = reinterpret_cast<double*>(dev + o_en);
  b->dst.stats = reinterpret_cast<int*>(dev + o_st);
  b->dst.phi = reinterpret_cast<float4*>(dev + o_phi);
  return b;
}

bool fits(const Staging* b, size_t npx, int L, int V, int ne) {
  return b->npx >= npx && b->L >= L && b->V >= V && b->ne >= ne;
}

void free_request(Request* r) {
  if (!r) return;
  free_staging(r->b);
  delete r;
}

void CUDART_CB on_step_done(void* p) {
  Step* st = static_cast<Step*>(p);
  st->t_done = clk::now();
  trk_server* sv = st->sv;
  {
    std::lock_guard<std::mutex> l(sv->sig_mu);
    sv->finished.push_back(st);
  }
  sv->cv_sig.notify_one();
}

void signal_work(trk_server* sv) {
  {
    std::lock_guard<std::mutex> l(sv->sig_mu);
    sv->work = true;
  }
  sv->cv_sig.notify_one();
}

// a step is done: its frames are collected by trk_server_wait (lock held)
void complete(trk_server* sv, Step* st) {
  for (Request* r : st->reqs) {
    r->state = 2;
    r->t_done = st->t_done;
    sv->lat.add(std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count());
    ++sv->completed;
    auto it = sv->sessions.find(r->s);
    if (it != sv->sessions.end() && it->second.inflight == r) it->second.inflight = nullptr;
    --sv->inflight;
  }
  ++sv->steps;
  sv->frames_in_steps += st->reqs.size();
  st->reqs.clear();
  if (st->bs) {
    st->busy = false;
  } else {
    delete st;
  }
}

// frames that could not be launched end at once with the error
void fail_requests(trk_server* sv, std::vector<Request*>& rs, trk_status e) {
  for (Request* r : rs) {
    r->status = e;
    r->state = 2;
    r->t_done = clk::now();
    auto it = sv->sessions.find(r->s);
    if (it != sv->sessions.end() && it->second.inflight == r) it->second.inflight = nullptr;
    --sv->inflight;
  }
  rs.clear();
}

void launch_session(trk_server* sv, trk_session* s, SessionSlot& sl) {
  Request* r = sl.pending.front();
  sl.pending.pop_front();
  r->state = 1;
  sl.inflight = r;
  ++sv->inflight;
  Step* st = new Step();
  st->sv = sv;
  st->reqs.push_back(r);
  trk_status e = trk::session_enqueue_frame(s, r->b->depth, &st->st);
  if (e == TRK_OK)
    e = trk::session_enqueue_results(s, r->b->theta, reinterpret_cast<float*>(r->b->phi), r->b->energy, r->b->stats);
  if (e == TRK_OK && cudaLaunchHostFunc(st->st, on_step_done, st) != cudaSuccess) e = TRK_ERR_CUDA;
  if (e != TRK_OK) {
    fail_requests(sv, st->reqs, e);
    delete st;
    sv->cv_done.notify_all();
  }
}

void launch_batched(trk_server* sv, Step* slot, std::vector<trk_session*>& ss) {
  std::vector<const float*> srcs;
  std::vector<trk::ResultDst> dst;
  for (trk_session* s : ss) {
    SessionSlot& sl = sv->sessions[s];
    Request* r = sl.pending.front();
    sl.pending.pop_front();
    r->state = 1;
    sl.inflight = r;
    ++sv->inflight;
    slot->reqs.push_back(r);
    srcs.push_back(r->b->depth_dev);
    dst.push_back(r->b->dst);
  }
  trk_status e = trk::batch_step_launch(slot->bs, ss.data(), (int)ss.size(), srcs.data(), dst.data(), slot->st);
  if (e == TRK_OK && cudaLaunchHostFunc(slot->st, on_step_done, slot) != cudaSuccess) e = TRK_ERR_CUDA;
  if (e != TRK_OK) {
    fail_requests(sv, slot->reqs, e);
    sv->cv_done.notify_all();
    return;
  }
  slot->busy = true;
}

// launches every frame that may start now (lock held)
void launch_ready(trk_server* sv) {
  const bool batched = sv->dispatch == TRK_SERVER_DISPATCH_BATCHED;
  for (auto& kv : sv->sessions) {
    if (sv->inflight >= sv->max_inflight) return;
    SessionSlot& sl = kv.second;
    if (sl.inflight || sl.pending.empty() || (batched && sl.batchable)) continue;
    launch_session(sv, kv.first, sl);
  }
  if (!batched) return;
  for (;;) {
    if (sv->inflight >= sv->max_inflight) return;
    Step* slot = nullptr;
    for (Step* s : sv->slots)
      if (!s->busy) {
        slot = s;
        break;
      }
    if (!slot) return;
    // the ready sessions, oldest waiting frame first; the step takes the class of the oldest
    std::vector<std::pair<clk::time_point, trk_session*>> ready;
    for (auto& kv : sv->sessions) {
      const SessionSlot& sl = kv.second;
      if (sl.batchable && !sl.inflight && !sl.pending.empty())
        ready.emplace_back(sl.pending.front()->t_submit, kv.first);
    }
    if (ready.empty()) return;
    std::sort(ready.begin(), ready.end(),
              [](const auto& a, const auto& b) { return a.first < b.first || (a.first == b.first && a.second < b.second); });
    const uint64_t key = sv->sessions[ready[0].second].key;
    const int room = std::min(sv->max_batch, sv->max_inflight - sv->inflight);
    std::vector<trk_session*> take;
    for (const auto& rd : ready)
      if ((int)take.size() < room && sv->sessions[rd.second].key == key) take.push_back(rd.second);
    // While another step runs, a small step waits for company: it goes once it holds its share of the
    // attached sessions (sessions / concurrent steps) or its oldest frame has waited max_wait_us; with
    // no step running it goes at once.  Eager small steps would keep the batches small.
    int running = 0, batchable = 0;
    for (Step* s2 : sv->slots) running += s2->busy;
    for (auto& kv : sv->sessions) batchable += kv.second.batchable && kv.second.key == key;
    const int share = std::min(room, (batchable + sv->n_slots - 1) / sv->n_slots);
    const clk::time_point due = ready[0].first + std::chrono::microseconds(sv->max_wait_us);
    if (running > 0 && (int)take.size() < share && clk::now() < due) {
      if (!sv->wake_set || due < sv->wake) {
        sv->wake = due;
        sv->wake_set = true;
      }
      return;
    }
    launch_batched(sv, slot, take);
  }
}

void worker_loop(trk_server* sv) {
  cudaSetDevice(sv->device);
  for (;;) {
    std::vector<Step*> fin;
    bool stop = false;
    clk::time_point wake{};
    bool timed = false;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      timed = sv->wake_set;
      wake = sv->wake;
    }
    {
      std::unique_lock<std::mutex> l(sv->sig_mu);
      auto pred = [&] { return !sv->finished.empty() || sv->work || sv->stop; };
      if (timed)
        sv->cv_sig.wait_until(l, wake, pred);
      else
        sv->cv_sig.wait(l, pred);
      fin.swap(sv->finished);
      sv->work = false;
      stop = sv->stop;
    }
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      for (Step* st : fin) complete(sv, st);
      sv->wake_set = false;
      if (!stop) launch_ready(sv);
    }
    if (!fin.empty()) sv->cv_done.notify_all();
    if (stop) return;
  }
}

// What the batched step slots may hold: each slot's buffer is at most twice its step's tables (rounded up
// to the granularity), a step's sessions are attached ones, and the reservation never shrinks (a slot
// keeps its buffer until a smaller step remakes it).
size_t step_reserve(const trk_server* sv, size_t step_sum) {
  if (sv->dispatch != TRK_SERVER_DISPATCH_BATCHED || step_sum == 0) return 0;
  return (size_t)sv->n_slots * ((2 * step_sum + sv->gran - 1) / sv->gran * sv->gran);
}

uint64_t class_key(const trk_params& p) {
  uint64_t k = (uint64_t)p.pose_iters;
  for (int v : {p.shape_iters, p.shape_sweeps, p.precision, p.shape_solver, p.association, p.mode})
    k = k * 1000003ull + (uint64_t)(v + 1);
  return k;
}

}  // namespace

extern "C" {

trk_status trk_server_create(size_t hbm_budget_bytes, int32_t max_inflight, trk_server** out) {
  if (!out || max_inflight < 0) return trk::set_error(TRK_ERR_INVALID_ARG, "trk_server_create: bad arguments");
  trk_server* sv = new trk_server();
  sv->budget = hbm_budget_bytes;
  sv->max_inflight = max_inflight;
  cudaGetDevice(&sv->device);
  if (const size_t g = trk::vmm_granularity()) sv->gran = g;
  sv->worker = std::thread(worker_loop, sv);
  *out = sv;
  return TRK_OK;
}

trk_status trk_server_configure(trk_server* sv, int32_t dispatch, int32_t max_batch, int32_t concurrent_steps,
                                int64_t max_wait_us) {
  if (!sv || (dispatch != TRK_SERVER_DISPATCH_BATCHED && dispatch != TRK_SERVER_DISPATCH_SESSION) || max_batch < 1 ||
      max_batch > 4096 || concurrent_steps < 1 || concurrent_steps > 16 || max_wait_us < 0)
    return trk::set_error(TRK_ERR_INVALID_ARG, "trk_server_configure: bad arguments");
  std::lock_guard<std::mutex> lk(sv->mu);
  if (!sv->sessions.empty() || !sv->attaching.empty() || !sv->slots.empty())
    return trk::set_error(TRK_ERR_INVALID_ARG, "trk_server_configure: call it before the first attach");
  sv->dispatch = dispatch;
  sv->max_batch = max_batch;
  sv->n_slots = concurrent_steps;
  sv->max_wait_us = max_wait_us;
  return TRK_OK;
}

trk_status trk_server_attach(trk_server* sv, trk_session* s) {
  if (!sv || !s) return trk::set_error(TRK_ERR_INVALID_ARG, "trk_server_attach: NULL argument");
  if (trk::session_device(s) != sv->device)
    return trk::set_error(TRK_ERR_INVALID_ARG, "trk_server_attach: session is on another device");
  const size_t arena = trk::session_device_bytes(s);
  size_t steps = 0;
  const bool was_resident = trk::session_resident(s);
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    // the session's arena, and the batched steps' buffers with its tables among theirs
    const bool batched = sv->dispatch == TRK_SERVER_DISPATCH_BATCHED && trk::session_params(s).mode == TRK_MODE_TRACK;
    steps = batched ? trk::batch_step_bytes_of(s) : 0;
    if (sv->sessions.count(s) || sv->attaching.count(s))
      return trk::set_error(TRK_ERR_INVALID_ARG, "trk_server_attach: already attached");
    const size_t peak = std::max(sv->step_peak, sv->step_sum + steps);
    if (sv->arena_used + arena + step_reserve(sv, peak) > sv->budget)
      return trk::set_error(TRK_ERR_NO_CAPACITY, "trk_server_attach: the session does not fit the HBM budget");
    sv->arena_used += arena;  // reserved while the device state is made
    sv->step_sum += steps;
    sv->step_peak = peak;
    sv->used = sv->arena_used + step_reserve(sv, sv->step_peak);
    sv->attaching[s] = true;
    if (sv->dispatch == TRK_SERVER_DISPATCH_BATCHED && sv->slots.empty()) {
      for (int k = 0; k < sv->n_slots; ++k) {
        Step* st = new Step();
        st->sv = sv;
        st->bs = trk::batch_step_create();
        if (!st->bs || cudaStreamCreateWithFlags(&st->st, cudaStreamNonBlocking) != cudaSuccess) {
          if (st->bs) trk::batch_step_destroy(st->bs, nullptr);
          delete st;
          break;
        }
        sv->slots.push_back(st);
      }
      if (sv->slots.empty()) {
        sv->arena_used -= arena;
        sv->step_sum -= steps;
        sv->used = sv->arena_used + step_reserve(sv, sv->step_peak);
        sv->attaching.erase(s);
        return trk::set_error(TRK_ERR_CUDA, "trk_server_attach: step stream creation failed");
      }
    }
  }
  trk_status e = was_resident ? TRK_OK : trk::session_restore(s);  // the device state, outside the lock
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->attaching.erase(s);
  if (e != TRK_OK) {
    sv->arena_used -= arena;
    sv->step_sum -= steps;
    sv->used = sv->arena_used + step_reserve(sv, sv->step_peak);
    return e;
  }
  SessionSlot& sl = sv->sessions[s];
  sl.bytes = arena;
  sl.step_bytes = steps;
  sl.restored = !was_resident;
  const trk_params& p = trk::session_params(s);
  sl.batchable = p.mode == TRK_MODE_TRACK;
  sl.key = class_key(p);
  return TRK_OK;
}

trk_status trk_server_detach(trk_server* sv, trk_session* s) {
  if (!sv || !s) return trk::set_error(TRK_ERR_INVALID_ARG, "trk_server_detach: NULL argument");
  bool evict = false;
  size_t bytes = 0, steps = 0;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->sessions.find(s);
    if (it == sv->sessions.end()) return trk::set_error(TRK_ERR_INVALID_ARG, "trk_server_detach: not attached");
    if (!it->second.pending.empty() || it->second.inflight)
      return trk::set_error(TRK_ERR_INVALID_ARG, "trk_server_detach: the session still has frames");
    for (Staging* b : it->second.spare) sv->pool.push_back(b);
    for (Step* st : sv->slots) trk::session_forget_stream(s, st->st);  // its frames there are done
    evict = it->second.restored;
    bytes = it->second.bytes;
    steps = it->second.step_bytes;
    sv->sessions.erase(it);
    sv->attaching[s] = true;  // until its device state is gone, the budget still holds it
  }
  const trk_status e = evict ? trk::session_evict(s) : TRK_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->attaching.erase(s);
    sv->arena_used -= bytes;
    sv->step_sum -= steps;
    sv->used = sv->arena_used + step_reserve(sv, sv->step_peak);
  }
  signal_work(sv);
  return e;
}

trk_status trk_server_submit(trk_server* sv, trk_session* s, const float* depth_m, uint64_t* ticket) {
  trk::NvtxRange nv("trk_server_submit");
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
    } else {
      for (size_t k = 0; k < sv->pool.size(); ++k)
        if (fits(sv->pool[k], npx, L, V, ne)) {
          r->b = sv->pool[k];
          sv->pool.erase(sv->pool.begin() + (long)k);
          break;
        }
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
      sv->pool.push_back(r->b);
      delete r;
      return trk::set_error(TRK_ERR_INVALID_ARG, "trk_server_submit: session not attached");
    }
    r->ticket = sv->next_ticket++;
    sv->requests[r->ticket] = r;
    it->second.pending.push_back(r);
    *ticket = r->ticket;
  }
  signal_work(sv);
  return TRK_OK;
}

trk_status trk_server_wait(trk_server* sv, uint64_t ticket, int64_t timeout_us, trk_result* out) {
  trk::NvtxRange nv("trk_server_wait");
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
      for (int i = 0; i < V; ++i) {
        out->offsets[3 * i] = b->phi[i].x;
        out->offsets[3 * i + 1] = b->phi[i].y;
        out->offsets[3 * i + 2] = b->phi[i].z;
      }
    out->n_assoc_px = b->stats[0];
    out->n_assoc_verts = b->stats[1];
  }
  lk.lock();  // the staging goes back to its session, or to the pool if the session left meanwhile
  auto it = sv->sessions.find(r->s);
  if (it != sv->sessions.end())
    it->second.spare.push_back(r->b);
  else
    sv->pool.push_back(r->b);
  r->b = nullptr;
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
  out->latency_p50_us = sv->lat.percentile(0.50);
  out->latency_p99_us = sv->lat.percentile(0.99);
  out->latency_max_us = sv->lat.max_us;
  out->steps = sv->steps;
  out->device_bytes_reserved = trk::vmm_bytes_held();
  out->mean_frames_per_step = sv->steps ? (double)sv->frames_in_steps / (double)sv->steps : 0.0;
  return TRK_OK;
}

void trk_server_destroy(trk_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> l(sv->sig_mu);
    sv->stop = true;
  }
  sv->cv_sig.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  // frames still on the GPU: wait for their streams (their host functions run before this returns)
  cudaDeviceSynchronize();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    for (Step* st : sv->finished) complete(sv, st);
    sv->finished.clear();
    for (auto& kv : sv->sessions) {
      for (Staging* b : kv.second.spare) free_staging(b);
      for (Step* st : sv->slots) trk::session_forget_stream(kv.first, st->st);
      if (kv.second.restored) trk::session_evict(kv.first);
    }
    for (Staging* b : sv->pool) free_staging(b);
    for (auto& kv : sv->requests) free_request(kv.second);
    for (Step* st : sv->slots) {
      trk::batch_step_destroy(st->bs, st->st);
      cudaStreamDestroy(st->st);
      delete st;
    }
  }
  delete sv;
}

}  // extern "C"
