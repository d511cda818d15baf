// schedule.cu -- how a set of sessions is stepped each frame, and the autotuner that chooses it (the
// schedule calls of trk.h).
//
// A schedule splits the sessions into `groups` work-balanced groups (largest first onto the lightest
// group).  A group of several sessions runs as one fused batch (one launch per stage over all its
// sessions), a group of one as the session's own frame graph; the groups run on concurrent streams
// joined to the caller's stream, so the stages of different groups overlap on the device.  groups = 1
// is one fused batch; groups = n is one graph per session.  The fused groups' association launches take
// assoc_blocks persistent blocks and tail_blocks queue-draining blocks.
//
// The autotuner times candidate schedules on real frames (CUDA events on the caller's stream), keeps the
// fastest, and stores it in a JSON cache keyed by the batch's size class, which later schedules of the
// same class read instead of tuning again.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/trk.h"
#include "trk_internal.cuh"

namespace trk {
const Dev& session_dev(const trk_session* s);
const trk_params& session_params(const trk_session* s);
void session_forget_stream(trk_session* s, cudaStream_t st);
trk_status batch_create(trk_session* const* sessions, int n, int assoc_blocks, int tail_blocks, trk_batch** out);
}  // namespace trk

using namespace trk;

struct trk_schedule {
  std::vector<trk_session*> sessions;
  trk_schedule_config cfg{};
  std::vector<std::vector<int>> groups;  // member indices per group
  std::vector<trk_batch*> batches;       // per group (nullptr for a group of one)
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;
  cudaEvent_t fork = nullptr;
  std::vector<const float*> ptrs;  // per-group depth pointers of the current frame
};

namespace {

double work_of(const trk_session* s) {
  const Dev& d = session_dev(s);
  return (double)d.V + 0.25 * (double)d.cam.W * d.cam.H;  // vertex passes dominate; pixels are cheaper
}

void release(trk_schedule* s) {
  for (trk_batch* b : s->batches)
    if (b) trk_batch_destroy(b);
  s->batches.clear();
  for (cudaStream_t st : s->streams) {  // the members' frames there end before the streams go
    cudaStreamSynchronize(st);
    for (trk_session* m : s->sessions) session_forget_stream(m, st);
  }
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  s->streams.clear();
  for (cudaEvent_t e : s->done) cudaEventDestroy(e);
  s->done.clear();
  if (s->fork) cudaEventDestroy(s->fork);
  s->fork = nullptr;
  s->groups.clear();
}

trk_status build(trk_schedule* s, const trk_schedule_config& c) {
  const int n = (int)s->sessions.size();
  if (c.groups < 1 || c.groups > n || c.assoc_blocks < 1 || c.tail_blocks < 1)
    return set_error(TRK_ERR_INVALID_ARG, "trk_schedule: groups must be in [1, n], block counts >= 1");
  release(s);
  s->cfg = c;
  // longest-processing-time partition: sessions by decreasing work, each onto the lightest group
  std::vector<int> order(n);
  for (int k = 0; k < n; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return work_of(s->sessions[a]) > work_of(s->sessions[b]); });
  s->groups.assign(c.groups, {});
  std::vector<double> load(c.groups, 0.0);
  for (int k : order) {
    const int g = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    s->groups[g].push_back(k);
    load[g] += work_of(s->sessions[k]);
  }
  for (auto& g : s->groups) std::sort(g.begin(), g.end());
  for (const auto& g : s->groups) {
    trk_batch* b = nullptr;
    if (g.size() > 1) {
      std::vector<trk_session*> members;
      for (int k : g) members.push_back(s->sessions[k]);
      const trk_status e = batch_create(members.data(), (int)members.size(), c.assoc_blocks, c.tail_blocks, &b);
      if (e != TRK_OK) {
        release(s);
        return e;
      }
    }
    s->batches.push_back(b);
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      if (st) cudaStreamDestroy(st);
      release(s);
      return set_error(TRK_ERR_CUDA, "trk_schedule: stream or event creation failed");
    }
    s->streams.push_back(st);
    s->done.push_back(ev);
  }
  if (cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming) != cudaSuccess) {
    release(s);
    return set_error(TRK_ERR_CUDA, "trk_schedule: event creation failed");
  }
  return TRK_OK;
}

trk_status step(trk_schedule* s, const float* const* d_depths, cudaStream_t st) {
  if (cudaEventRecord(s->fork, st) != cudaSuccess) return set_error(TRK_ERR_CUDA, "trk_schedule: event record failed");
  for (size_t g = 0; g < s->groups.size(); ++g) {
    cudaStream_t gs = s->streams[g];
    if (cudaStreamWaitEvent(gs, s->fork, 0) != cudaSuccess)
      return set_error(TRK_ERR_CUDA, "trk_schedule: stream wait failed");
    trk_status e;
    if (s->batches[g]) {
      s->ptrs.clear();
      for (int k : s->groups[g]) s->ptrs.push_back(d_depths[k]);
      e = trk_batch_track_device(s->batches[g], s->ptrs.data(), gs);
    } else {
      const int k = s->groups[g][0];
      e = trk_track_frame_device(s->sessions[k], d_depths[k], gs);
    }
    if (e != TRK_OK) return e;
    if (cudaEventRecord(s->done[g], gs) != cudaSuccess || cudaStreamWaitEvent(st, s->done[g], 0) != cudaSuccess)
      return set_error(TRK_ERR_CUDA, "trk_schedule: join failed");
  }
  return TRK_OK;
}

// ---- the tuning cache: a JSON object {"<size class>": {"groups": G, "assoc_blocks": A, "tail_blocks": T,
// "ms_per_step": x}, ...}, read and written whole --------------------------------------------------------
std::map<std::string, std::string> read_cache(const char* path) {
  std::map<std::string, std::string> out;
  if (!path) return out;
  FILE* f = std::fopen(path, "rb");
  if (!f) return out;
  std::string txt;
  char buf[4096];
  size_t r;
  while ((r = std::fread(buf, 1, sizeof(buf), f)) > 0) txt.append(buf, r);
  std::fclose(f);
  size_t p = txt.find('{');
  if (p == std::string::npos) return out;
  ++p;
  for (;;) {
    const size_t k0 = txt.find('"', p);
    if (k0 == std::string::npos) break;
    const size_t k1 = txt.find('"', k0 + 1);
    const size_t o0 = txt.find('{', k1);
    const size_t o1 = txt.find('}', o0);
    if (k1 == std::string::npos || o0 == std::string::npos || o1 == std::string::npos) break;
    out[txt.substr(k0 + 1, k1 - k0 - 1)] = txt.substr(o0, o1 - o0 + 1);
    p = o1 + 1;
  }
  return out;
}

bool field(const std::string& obj, const char* name, double& v) {
  const std::string key = std::string("\"") + name + "\"";
  const size_t p = obj.find(key);
  if (p == std::string::npos) return false;
  const size_t c = obj.find(':', p + key.size());
  if (c == std::string::npos) return false;
  char* end = nullptr;
  v = std::strtod(obj.c_str() + c + 1, &end);
  return end != obj.c_str() + c + 1;
}

bool write_cache(const char* path, const std::map<std::string, std::string>& entries) {
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return false;
  std::fputs("{\n", f);
  size_t i = 0;
  for (const auto& kv : entries)
    std::fprintf(f, "  \"%s\": %s%s\n", kv.first.c_str(), kv.second.c_str(), ++i < entries.size() ? "," : "");
  std::fputs("}\n", f);
  const bool ok = std::fclose(f) == 0;
  return ok && std::rename(tmp.c_str(), path) == 0;
}

std::string entry_text(const trk_schedule_config& c, double ms) {
  char buf[256];
  std::snprintf(buf, sizeof(buf), "{\"groups\": %d, \"assoc_blocks\": %d, \"tail_blocks\": %d, \"ms_per_step\": %.4f}",
                c.groups, c.assoc_blocks, c.tail_blocks, ms);
  return buf;
}

trk_schedule_config default_config(int n) {
  trk_schedule_config c{};
  c.groups = 1;
  c.assoc_blocks = kAssocBlocksPerSM * 152;
  c.tail_blocks = 2 * 152;
  (void)n;
  return c;
}

}  // namespace

extern "C" {

trk_status trk_schedule_signature(trk_session* const* sessions, int32_t n, char* out, size_t out_size) {
  if (!sessions || n < 1 || !out || out_size < 8) return set_error(TRK_ERR_INVALID_ARG, "trk_schedule_signature: bad arguments");
  double V = 0, px = 0;
  int L = 0, prec = session_params(sessions[0]).precision;
  for (int k = 0; k < n; ++k) {
    if (!sessions[k]) return set_error(TRK_ERR_INVALID_ARG, "trk_schedule_signature: NULL session");
    const Dev& d = session_dev(sessions[k]);
    V += d.V;
    px += (double)d.cam.W * d.cam.H;
    L = std::max(L, d.L);
  }
  // size class: session count, precision, total vertices and pixels to two significant digits, links
  auto two = [](double x) {
    if (x <= 0) return 0.0;
    const double e = std::pow(10.0, std::floor(std::log10(x)) - 1);
    return std::round(x / e) * e;
  };
  std::snprintf(out, out_size, "n%d_p%d_v%.0f_px%.0f_L%d", n, prec, two(V), two(px), L);
  return TRK_OK;
}

trk_status trk_tuning_cache_lookup(const char* path, const char* signature, trk_schedule_config* out, double* ms) {
  if (!path || !signature || !out) return set_error(TRK_ERR_INVALID_ARG, "trk_tuning_cache_lookup: NULL argument");
  const auto entries = read_cache(path);
  const auto it = entries.find(signature);
  if (it == entries.end()) return set_error(TRK_ERR_INVALID_ARG, "trk_tuning_cache_lookup: no entry for this size class");
  double g = 0, a = 0, t = 0, m = 0;
  if (!field(it->second, "groups", g) || !field(it->second, "assoc_blocks", a) || !field(it->second, "tail_blocks", t))
    return set_error(TRK_ERR_INVALID_ARG, "trk_tuning_cache_lookup: malformed entry");
  out->groups = (int32_t)g;
  out->assoc_blocks = (int32_t)a;
  out->tail_blocks = (int32_t)t;
  if (ms) *ms = field(it->second, "ms_per_step", m) ? m : 0.0;
  return TRK_OK;
}

trk_status trk_tuning_cache_store(const char* path, const char* signature, const trk_schedule_config* cfg, double ms) {
  if (!path || !signature || !cfg) return set_error(TRK_ERR_INVALID_ARG, "trk_tuning_cache_store: NULL argument");
  if (std::strchr(signature, '"') || std::strchr(signature, '\\'))
    return set_error(TRK_ERR_INVALID_ARG, "trk_tuning_cache_store: bad signature");
  auto entries = read_cache(path);
  entries[signature] = entry_text(*cfg, ms);
  if (!write_cache(path, entries)) return set_error(TRK_ERR_INVALID_ARG, "trk_tuning_cache_store: cannot write the cache file");
  return TRK_OK;
}

trk_status trk_schedule_create(trk_session* const* sessions, int32_t n, const trk_schedule_config* cfg,
                               const char* cache_path, trk_schedule** out) {
  if (!sessions || n < 1 || !out) return set_error(TRK_ERR_INVALID_ARG, "trk_schedule_create: bad arguments");
  for (int k = 0; k < n; ++k)
    if (!sessions[k]) return set_error(TRK_ERR_INVALID_ARG, "trk_schedule_create: NULL session");
  trk_schedule_config c = default_config(n);
  if (cfg) {
    c = *cfg;
  } else if (cache_path) {
    char sig[256];
    trk_schedule_config cached{};
    if (trk_schedule_signature(sessions, n, sig, sizeof(sig)) == TRK_OK &&
        trk_tuning_cache_lookup(cache_path, sig, &cached, nullptr) == TRK_OK && cached.groups >= 1 &&
        cached.groups <= n)
      c = cached;
  }
  trk_schedule* s = new trk_schedule();
  s->sessions.assign(sessions, sessions + n);
  const trk_status e = build(s, c);
  if (e != TRK_OK) {
    delete s;
    return e;
  }
  *out = s;
  return TRK_OK;
}

trk_status trk_schedule_track_device(trk_schedule* s, const float* const* d_depths, void* cuda_stream) {
  NvtxRange nv("trk_schedule_track_device");
  if (!s || !d_depths) return set_error(TRK_ERR_INVALID_ARG, "trk_schedule_track_device: NULL argument");
  return step(s, d_depths, (cudaStream_t)cuda_stream);
}

trk_status trk_schedule_get_config(const trk_schedule* s, trk_schedule_config* out) {
  if (!s || !out) return set_error(TRK_ERR_INVALID_ARG, "trk_schedule_get_config: NULL argument");
  *out = s->cfg;
  return TRK_OK;
}

constexpr int kSettleSteps = 4;  // frames tracked before the autotuner's timed trials

trk_status trk_schedule_autotune(trk_schedule* s, const float* const* d_depths, int32_t reps, const char* cache_path,
                                 trk_schedule_config* chosen, double* ms_per_step) {
  if (!s || !d_depths || reps < 1) return set_error(TRK_ERR_INVALID_ARG, "trk_schedule_autotune: bad arguments");
  const int n = (int)s->sessions.size();
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    return set_error(TRK_ERR_CUDA, "trk_schedule_autotune: stream or event creation failed");
  auto measure = [&](const trk_schedule_config& c, double& ms) -> trk_status {
    trk_status e = build(s, c);
    if (e != TRK_OK) return e;
    if ((e = step(s, d_depths, st)) != TRK_OK) return e;  // warm-up (first graph launches)
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps; ++r)
      if ((e = step(s, d_depths, st)) != TRK_OK) return e;
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) return set_error(TRK_ERR_CUDA, "trk_schedule_autotune: timing failed");
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    ms = t / reps;
    return TRK_OK;
  };
  // coordinate search: the group count first (default blocks), then the association block counts.  The
  // trials all track the same frame, so the sessions first settle on it under the default schedule: every
  // candidate is then timed from the same converged state (without this, the first candidates would be
  // timed on the frame's harder first visits and the later ones would be favoured).
  trk_schedule_config best = default_config(n);
  double best_ms = 1e30;
  trk_status err = build(s, best);
  for (int w = 0; err == TRK_OK && w < kSettleSteps; ++w) err = step(s, d_depths, st);
  if (err != TRK_OK) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    return err;
  }
  std::vector<int> gs;
  for (int g : {1, 2, 4, 8, 16, 32})
    if (g < n) gs.push_back(g);
  gs.push_back(n);
  for (int g : gs) {
    trk_schedule_config c = best;
    c.groups = g;
    double ms = 0;
    if ((err = measure(c, ms)) != TRK_OK) break;
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  if (err == TRK_OK && best.groups < n) {
    const trk_schedule_config base = best;
    for (int a : {2 * 152, kAssocBlocksPerSM * 152, 2 * kAssocBlocksPerSM * 152})
      for (int t : {152, 2 * 152, 4 * 152}) {
        if (a == base.assoc_blocks && t == base.tail_blocks) continue;
        trk_schedule_config c = base;
        c.assoc_blocks = a;
        c.tail_blocks = t;
        double ms = 0;
        if ((err = measure(c, ms)) != TRK_OK) break;
        if (ms < best_ms) {
          best_ms = ms;
          best = c;
        }
      }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  if (err != TRK_OK) return err;
  if ((err = build(s, best)) != TRK_OK) return err;
  if (chosen) *chosen = best;
  if (ms_per_step) *ms_per_step = best_ms;
  if (cache_path) {
    char sig[256];
    if ((err = trk_schedule_signature(s->sessions.data(), n, sig, sizeof(sig))) != TRK_OK) return err;
    if ((err = trk_tuning_cache_store(cache_path, sig, &best, best_ms)) != TRK_OK) return err;
  }
  return TRK_OK;
}

void trk_schedule_destroy(trk_schedule* s) {
  if (!s) return;
  for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
  release(s);
  delete s;
}

}  // extern "C"
