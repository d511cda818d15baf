// batch.cu -- many tracking sessions stepped together (the batch calls of trk.h).
//
// Every stage of a frame (skinning, z-buffer, visibility, association, [J r]^T [J r], the LM solve and
// acceptance, the shape step) runs as ONE kernel launch over the blocks of all sessions: a per-stage
// table maps each block to (session, block position in that session's grid), and the block reads its
// session's descriptor from a device array.  A frame of the whole batch is one CUDA graph of the same
// ~110 launches a single session needs, however many sessions there are, and the sessions' blocks share
// each launch's waves (small sessions fill the gaps of large ones).  Each session computes exactly what
// it computes alone: blocks of different sessions touch disjoint buffers, and every per-session
// reduction keeps its fixed order.
#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/trk.h"
#include "trk_internal.cuh"

namespace trk {
const Dev& session_dev(const trk_session* s);
const trk_params& session_params(const trk_session* s);
int session_device(const trk_session* s);
void session_set_last_stream(trk_session* s, cudaStream_t st);
bool session_resident(const trk_session* s);
unsigned session_generation(const trk_session* s);
}  // namespace trk

using namespace trk;

namespace {

// kJtj1..kJtj5: the [J r] blocks of the sessions with tile width class ceil(NP / 16) = 1..5; kRows: the
// [J r] blocks of every session (the candidate energies read their rows)
enum Kind { kSkin, kTris, kVerts, kAssoc, kJtj1, kJtj2, kJtj3, kJtj4, kJtj5, kReduce, kLm, kRows, kKinds };
constexpr int kSrcSlots = 4;
constexpr int kMaxBatch = 4096;  // the tail's prefix kernel scans up to 1024 x 4 sessions

struct Table {
  int4* d_map = nullptr;
  int n = 0;
};

}  // namespace

struct trk_batch {
  std::vector<trk_session*> sessions;
  std::vector<unsigned> generations;  // each member's device-state generation when the batch was built
  int device = 0;
  int pose_iters = 0, shape_iters = 0, shape_sweeps = 0, precision = 0, shape_solver = 0;
  int max_links = 0, max_np = 0;
  int assoc_blocks = kAssocBlocksPerSM * 152;  // persistent association blocks
  int tail_blocks = 304;      // association-tail blocks (shared by all sessions' queues)
  Dev* d_devs = nullptr;
  unsigned* d_ctl = nullptr;  // [0] association units of the frame, [1] unused, [2] tail counter
  unsigned* d_prefix = nullptr;  // [n + 1] queued pixels before each session
  AssocUnit* d_tiles = nullptr;  // association units of the frame (up to 32 valid pixels of a tile each)
  Table tables[kKinds];
  const float** d_srcs = nullptr;  // device copy of the per-session depth pointers of the current frame
  const float** h_srcs = nullptr;  // pinned, kSrcSlots slots of one pointer per session
  cudaEvent_t src_ev[4] = {};      // the copy out of each slot has been done
  int src_slot = 0;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t graph = nullptr;
};

namespace {

BatchGrid grid_of(const trk_batch* b, Kind k) { return BatchGrid{b->d_devs, b->tables[k].d_map}; }

int reduce_threads_of(const trk_batch* b) {
  int w = 1;
  for (trk_session* s : b->sessions) w = std::max(w, reduce_warps(session_dev(s).nblk_rows));
  return 32 * w;
}

// The members' device state is still the one the batch's tables and graph point into.
bool members_current(const trk_batch* b) {
  for (size_t k = 0; k < b->sessions.size(); ++k)
    if (!session_resident(b->sessions[k]) || session_generation(b->sessions[k]) != b->generations[k]) return false;
  return true;
}

// Blocks of session s in the launches of kind k.
void blocks_of(const Dev& d, Kind k, int& gx, int& gy) {
  const int npx = d.cam.W * d.cam.H;
  gy = 1;
  switch (k) {
    case kSkin: gx = std::max((d.V + 255) / 256, (npx + 2047) / 2048); break;  // also clears the pixel buffers
    case kTris: gx = (d.F + 255) / 256; break;
    case kVerts: gx = d.nblk_v; break;
    case kAssoc: gx = (d.cam.W + 15) / 16; gy = (d.cam.H + 15) / 16; break;
    case kJtj1: case kJtj2: case kJtj3: case kJtj4: case kJtj5:
      gx = (d.NP + 15) / 16 == k - kJtj1 + 1 ? d.nblk_rows : 0;
      break;
    case kReduce: gx = (d.NP * (d.NP + 1) / 2 + 31) / 32; break;  // the upper triangle
    case kRows: gx = d.nblk_rows; break;
    default: gx = kCandidates; break;  // kLm
  }
}

// One batched frame over a set of sessions: the block tables, the sessions' descriptors and the scratch
// of the association, wherever they live (a trk_batch's own buffers or a server step's).
struct FrameView {
  int B = 0, P = 0, S = 0, sweeps = 0, solver = 0, precision = 0, max_links = 0;
  int assoc_blocks = 0, tail_blocks = 0;
  const Dev* d_devs = nullptr;
  Table tables[kKinds];
  unsigned* d_ctl = nullptr;        // [3]
  unsigned* d_prefix = nullptr;     // [B + 1]
  AssocUnit* d_tiles = nullptr;     // [kUnitsPerTile tables[kAssoc].n]
  const float* const* d_srcs = nullptr;  // [B] depth of each session (device-readable)
  const Dev* const* host_devs = nullptr;  // [B] the sessions' descriptors on the host
  int reduce_threads = 32;                // the reduction's block: the largest need of the sessions
};

int reduce_threads_for(const Dev* const* hd, int n) {
  int w = 1;
  for (int k = 0; k < n; ++k) w = std::max(w, reduce_warps(hd[k]->nblk_rows));
  return 32 * w;
}

BatchGrid grid_of(const FrameView& v, Kind k) { return BatchGrid{v.d_devs, v.tables[k].d_map}; }

void enqueue_frame_view(const FrameView& v, cudaStream_t st) {
  const int B = v.B, P = v.P, S = v.S, L = v.max_links;
  cudaMemsetAsync(v.d_ctl, 0, sizeof(unsigned) * 3, st);
  launch_gather_depth_b(grid_of(v, kAssoc), v.tables[kAssoc].n, v.d_srcs, v.d_tiles, v.d_ctl, st);
  int cur = 0;
  auto geometry = [&]() {
    NvtxRange nv("skin, z-buffer, visibility, association");
    launch_skin_b(grid_of(v, kSkin), v.tables[kSkin].n, L, cur, v.d_ctl, st);
    launch_raster_b(grid_of(v, kTris), v.tables[kTris].n, st);
    launch_visibility_b(grid_of(v, kVerts), v.tables[kVerts].n, st);
    launch_associate_b(v.d_devs, B, v.d_tiles, v.d_ctl, v.d_prefix, v.assoc_blocks, v.tail_blocks, st);
  };
  for (int it = 0; it < P; ++it) {
    geometry();
    BatchGrid gj[5];
    int nj[5];
    for (int t = 0; t < 5; ++t) {
      gj[t] = grid_of(v, (Kind)(kJtj1 + t));
      nj[t] = v.tables[kJtj1 + t].n;
    }
    NvtxRange nv("normal equations, LM step");
    launch_normal_equations_b(gj, nj, grid_of(v, kReduce), v.tables[kReduce].n, L, v.precision, cur, it, st,
                              v.reduce_threads);
    launch_lm_b(grid_of(v, kLm), v.tables[kLm].n, grid_of(v, kRows), v.tables[kRows].n, L, cur, st);
  }
  for (int it = 0; it < S; ++it) {
    geometry();
    NvtxRange nv("shape step");
    cur = launch_shape_b(grid_of(v, kVerts), v.tables[kVerts].n, L, v.sweeps, v.solver, cur, P + it, st);
  }
  if (cur != 0)
    for (int k = 0; k < B; ++k) {
      const Dev& d = *v.host_devs[k];
      cudaMemcpyAsync(d.phi[0], d.phi[cur], sizeof(float4) * d.V, cudaMemcpyDeviceToDevice, st);
    }
}

FrameView view_of(const trk_batch* b, const std::vector<const Dev*>& host_devs) {
  FrameView v;
  v.B = (int)b->sessions.size();
  v.P = b->pose_iters;
  v.S = b->shape_iters;
  v.sweeps = b->shape_sweeps;
  v.solver = b->shape_solver;
  v.precision = b->precision;
  v.max_links = b->max_links;
  v.assoc_blocks = b->assoc_blocks;
  v.tail_blocks = b->tail_blocks;
  v.d_devs = b->d_devs;
  for (int k = 0; k < kKinds; ++k) v.tables[k] = b->tables[k];
  v.d_ctl = b->d_ctl;
  v.d_prefix = b->d_prefix;
  v.d_tiles = b->d_tiles;
  v.d_srcs = b->d_srcs;
  v.host_devs = host_devs.data();
  v.reduce_threads = reduce_threads_for(host_devs.data(), v.B);
  return v;
}

void enqueue_batch_frame(trk_batch* b, cudaStream_t st) {
  std::vector<const Dev*> hd;
  for (trk_session* s : b->sessions) hd.push_back(&session_dev(s));
  enqueue_frame_view(view_of(b, hd), st);
}

void free_batch(trk_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (Table& t : b->tables) cudaFree(t.d_map);
  cudaFree(b->d_devs);
  cudaFree(b->d_ctl);
  cudaFree(b->d_prefix);
  cudaFree(b->d_tiles);
  cudaFree(b->d_srcs);
  for (cudaEvent_t e : b->src_ev)
    if (e) {
      cudaEventSynchronize(e);
      cudaEventDestroy(e);
    }
  cudaFreeHost(b->h_srcs);
  delete b;
}

#define BCK(call)                                                                 \
  do {                                                                            \
    const cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess) {                                                      \
      free_batch(b);                                                              \
      return set_error(e_ == cudaErrorMemoryAllocation ? TRK_ERR_OOM : TRK_ERR_CUDA, \
                       cudaGetErrorString(e_));                                   \
    }                                                                             \
  } while (0)

}  // namespace

namespace trk {

// trk_batch_create with the association's launch sizes: assoc_blocks persistent tile blocks and
// tail_blocks queue-draining blocks (the schedule's tunables).
trk_status batch_create(trk_session* const* sessions, int n_sessions, int assoc_blocks, int tail_blocks,
                        trk_batch** out) {
  if (!sessions || n_sessions < 1 || n_sessions > kMaxBatch || !out || assoc_blocks < 1 || tail_blocks < 1)
    return set_error(TRK_ERR_INVALID_ARG, "trk_batch_create: bad arguments (1 <= n_sessions <= 4096)");
  trk_batch* b = new trk_batch();
  b->assoc_blocks = assoc_blocks;
  b->tail_blocks = tail_blocks;
  const trk_params& p0 = session_params(sessions[0]);
  b->device = session_device(sessions[0]);
  b->pose_iters = p0.pose_iters;
  b->shape_iters = p0.shape_iters;
  b->shape_sweeps = p0.shape_sweeps;
  b->precision = p0.precision;
  b->shape_solver = p0.shape_solver;
  for (int k = 0; k < n_sessions; ++k) {
    trk_session* s = sessions[k];
    if (!s) {
      free_batch(b);
      return set_error(TRK_ERR_INVALID_ARG, "trk_batch_create: NULL session");
    }
    for (int j = 0; j < k; ++j)
      if (sessions[j] == s) {
        free_batch(b);
        return set_error(TRK_ERR_INVALID_ARG, "trk_batch_create: a session appears twice");
      }
    if (!session_resident(s)) {
      free_batch(b);
      return set_error(TRK_ERR_INVALID_ARG, "trk_batch_create: a session is evicted (trk_session_restore first)");
    }
    const trk_params& p = session_params(s);
    if (p.mode != TRK_MODE_TRACK) {
      free_batch(b);
      return set_error(TRK_ERR_INVALID_ARG, "trk_batch_create: batched sessions must be in TRK_MODE_TRACK");
    }
    if (session_device(s) != b->device || p.pose_iters != b->pose_iters || p.shape_iters != b->shape_iters ||
        p.shape_sweeps != b->shape_sweeps || p.precision != b->precision || p.shape_solver != b->shape_solver ||
        p.association != session_params(sessions[0]).association) {
      free_batch(b);
      return set_error(TRK_ERR_INVALID_ARG,
                       "trk_batch_create: sessions differ in device, schedule, precision, shape solver or association");
    }
    const Dev& d = session_dev(s);
    b->max_links = std::max(b->max_links, d.L);
    b->max_np = std::max(b->max_np, d.NP);
    b->sessions.push_back(s);
    b->generations.push_back(session_generation(s));
  }
  int cur_dev = 0;
  cudaGetDevice(&cur_dev);
  if (cur_dev != b->device) {
    free_batch(b);
    return set_error(TRK_ERR_INVALID_ARG, "trk_batch_create: the sessions' device is not the current device");
  }
  ensure_configured();
  std::vector<Dev> devs;
  for (trk_session* s : b->sessions) devs.push_back(session_dev(s));
  BCK(cudaMalloc(&b->d_devs, sizeof(Dev) * devs.size()));
  BCK(cudaMemcpy(b->d_devs, devs.data(), sizeof(Dev) * devs.size(), cudaMemcpyHostToDevice));
  for (int k = 0; k < kKinds; ++k) {
    std::vector<int4> map;
    for (int s = 0; s < (int)devs.size(); ++s) {
      int gx = 0, gy = 0;
      blocks_of(devs[s], (Kind)k, gx, gy);
      for (int y = 0; y < gy; ++y)
        for (int x = 0; x < gx; ++x) map.push_back(make_int4(s, x, y, gx));
    }
    b->tables[k].n = (int)map.size();
    if (!map.empty()) {
      BCK(cudaMalloc(&b->tables[k].d_map, sizeof(int4) * map.size()));
      BCK(cudaMemcpy(b->tables[k].d_map, map.data(), sizeof(int4) * map.size(), cudaMemcpyHostToDevice));
    }
  }
  BCK(cudaMalloc(&b->d_ctl, sizeof(unsigned) * 3));
  BCK(cudaMalloc(&b->d_prefix, sizeof(unsigned) * (n_sessions + 1)));
  BCK(cudaMalloc(&b->d_tiles, sizeof(AssocUnit) * kUnitsPerTile * std::max(b->tables[kAssoc].n, 1)));
  BCK(cudaMalloc(&b->d_srcs, sizeof(float*) * devs.size()));
  BCK(cudaMallocHost(&b->h_srcs, sizeof(float*) * devs.size() * kSrcSlots));
  for (cudaEvent_t& e : b->src_ev) BCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  BCK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  enqueue_batch_frame(b, b->cap);
  BCK(cudaStreamEndCapture(b->cap, &g));
  const cudaError_t e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  BCK(e);
  *out = b;
  return TRK_OK;
}

// ---- one batched frame over a varying set of sessions (the frame server's batched dispatch) --------
//
// Unlike a trk_batch (fixed members, one captured graph), a BatchStep launches the ~110 stage kernels of
// one frame directly, for whichever sessions have a frame ready.  Its tables, descriptors, depth and
// result pointers travel in one host-to-device copy from a pinned mirror; depth is read and results are
// written straight from / into host-mapped pinned memory (zero copy over the chip-to-chip link), so a
// step costs its launches, one small upload and no per-session copies.

__global__ void __launch_bounds__(256) k_results_b(BatchGrid g, const ResultDst* __restrict__ dst) {
  const int4 m = g.map[blockIdx.x];
  const Dev& d = g.devs[m.x];
  const ResultDst o = dst[m.x];
  const int i = m.y * 256 + threadIdx.x;
  if (i < d.V) o.phi[i] = d.phi[0][i];
  if (m.y == 0) {
    for (int t = threadIdx.x; t < d.L; t += blockDim.x) o.theta[t] = d.theta[t];
    for (int t = threadIdx.x; t < d.pose_iters + d.shape_iters; t += blockDim.x) o.energy[t] = d.energy[t];
    if (threadIdx.x < 4) o.stats[threadIdx.x] = d.stats[threadIdx.x];
  }
}

struct BatchStep {
  VmmBlock d_block;       // device: [upload part | ctl, prefix, tiles]
  char* d_buf = nullptr;
  char* h_buf = nullptr;  // pinned mirror of the upload part
  size_t d_cap = 0, h_cap = 0;
  cudaEvent_t uploaded = nullptr;  // the last upload out of h_buf has been done
};

BatchStep* batch_step_create() {
  BatchStep* bs = new BatchStep();
  if (cudaEventCreateWithFlags(&bs->uploaded, cudaEventDisableTiming) != cudaSuccess) {
    delete bs;
    return nullptr;
  }
  return bs;
}

void batch_step_destroy(BatchStep* bs, cudaStream_t st) {
  if (!bs) return;
  cudaEventSynchronize(bs->uploaded);
  cudaStreamSynchronize(st);
  vmm_free(&bs->d_block);
  if (bs->h_buf) cudaFreeHost(bs->h_buf);
  cudaEventDestroy(bs->uploaded);
  delete bs;
}

namespace {
size_t align16(size_t x) { return (x + 15) & ~size_t(15); }
}  // namespace

// Device bytes one session adds to a step's buffer: its descriptor, pointers, block-table entries and
// tiles (each region 16-byte aligned, hence the slack).
size_t batch_step_bytes_of(const trk_session* s) {
  const Dev& d = session_dev(s);
  size_t n = sizeof(Dev) + sizeof(float*) + sizeof(ResultDst) + sizeof(unsigned) + 16 * (kKinds + 4);
  for (int k = 0; k < kKinds; ++k) {
    int gx = 0, gy = 0;
    blocks_of(d, (Kind)k, gx, gy);
    n += sizeof(int4) * (size_t)gx * gy;
  }
  int gx = 0, gy = 0;
  blocks_of(d, kAssoc, gx, gy);
  return n + sizeof(AssocUnit) * kUnitsPerTile * (size_t)gx * gy;  // the step's list of association units
}

trk_status batch_step_launch(BatchStep* bs, trk_session* const* ss, int n, const float* const* srcs,
                             const ResultDst* dst, cudaStream_t st) {
  NvtxRange range("server batched step");
  if (!bs || !ss || n < 1 || n > kMaxBatch || !srcs || !dst)
    return set_error(TRK_ERR_INVALID_ARG, "batch step: bad arguments");
  const trk_params& p0 = session_params(ss[0]);
  int max_links = 0;
  std::vector<const Dev*> hd(n);
  for (int k = 0; k < n; ++k) {
    const trk_params& p = session_params(ss[k]);
    if (!session_resident(ss[k])) return set_error(TRK_ERR_INVALID_ARG, "batch step: a session is evicted");
    if (p.mode != TRK_MODE_TRACK || p.pose_iters != p0.pose_iters || p.shape_iters != p0.shape_iters ||
        p.shape_sweeps != p0.shape_sweeps || p.precision != p0.precision || p.shape_solver != p0.shape_solver ||
        p.association != p0.association)
      return set_error(TRK_ERR_INVALID_ARG, "batch step: sessions of different schedules, precision or mode");
    hd[k] = &session_dev(ss[k]);
    max_links = std::max(max_links, hd[k]->L);
  }
  // the block tables of this set of sessions
  std::vector<int4> maps[kKinds + 1];  // kKinds: the result kernel's (the vertex blocks)
  for (int k = 0; k < kKinds; ++k)
    for (int q = 0; q < n; ++q) {
      int gx = 0, gy = 0;
      blocks_of(*hd[q], (Kind)k, gx, gy);
      for (int y = 0; y < gy; ++y)
        for (int x = 0; x < gx; ++x) maps[k].push_back(make_int4(q, x, y, gx));
    }
  // layout: devs | srcs | dst | maps ... (uploaded) | ctl | prefix | tiles (device only)
  size_t off = 0;
  const size_t o_devs = off; off = align16(off + sizeof(Dev) * n);
  const size_t o_srcs = off; off = align16(off + sizeof(float*) * n);
  const size_t o_dst = off; off = align16(off + sizeof(ResultDst) * n);
  size_t o_map[kKinds];
  for (int k = 0; k < kKinds; ++k) {
    o_map[k] = off;
    off = align16(off + sizeof(int4) * maps[k].size());
  }
  const size_t upload = off;
  const size_t o_ctl = off; off = align16(off + sizeof(unsigned) * 4);
  const size_t o_prefix = off; off = align16(off + sizeof(unsigned) * (n + 1));
  const size_t o_tiles = off; off = align16(off + sizeof(AssocUnit) * kUnitsPerTile * std::max<size_t>(maps[kAssoc].size(), 1));
  const size_t total = off;
  // the previous upload out of the pinned mirror has been done
  cudaError_t e = cudaEventSynchronize(bs->uploaded);
  // remade at this step's size (rounded to the allocation granularity) when it needs more, or less than
  // half, so that the buffer holds at most twice what a step of these sessions needs; the slot's last step
  // has completed, so the old block is idle
  if (e == cudaSuccess && (total > bs->d_cap || 2 * total < bs->d_cap)) {
    e = cudaStreamSynchronize(st);
    vmm_free(&bs->d_block);
    bs->d_buf = nullptr;
    bs->d_cap = 0;
    if (e == cudaSuccess) e = vmm_alloc(total, &bs->d_block);
    if (e == cudaSuccess) {
      bs->d_buf = static_cast<char*>(bs->d_block.ptr);
      bs->d_cap = bs->d_block.size;
    }
  }
  if (e == cudaSuccess && upload > bs->h_cap) {  // pinned host memory: grown only
    if (bs->h_buf) cudaFreeHost(bs->h_buf);
    bs->h_buf = nullptr;
    bs->h_cap = 0;
    e = cudaMallocHost(reinterpret_cast<void**>(&bs->h_buf), 2 * upload);
    if (e == cudaSuccess) bs->h_cap = 2 * upload;
  }
  if (e != cudaSuccess)
    return set_error(e == cudaErrorMemoryAllocation ? TRK_ERR_OOM : TRK_ERR_CUDA, cudaGetErrorString(e));
  char* h = bs->h_buf;
  for (int k = 0; k < n; ++k) std::memcpy(h + o_devs + sizeof(Dev) * k, hd[k], sizeof(Dev));
  std::memcpy(h + o_srcs, srcs, sizeof(float*) * n);
  std::memcpy(h + o_dst, dst, sizeof(ResultDst) * n);
  for (int k = 0; k < kKinds; ++k)
    if (!maps[k].empty()) std::memcpy(h + o_map[k], maps[k].data(), sizeof(int4) * maps[k].size());
  e = cudaMemcpyAsync(bs->d_buf, h, upload, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(bs->uploaded, st);
  if (e != cudaSuccess) return set_error(TRK_ERR_CUDA, cudaGetErrorString(e));
  char* dbuf = bs->d_buf;
  FrameView v;
  v.B = n;
  v.P = p0.pose_iters;
  v.S = p0.shape_iters;
  v.sweeps = p0.shape_sweeps;
  v.solver = p0.shape_solver;
  v.precision = p0.precision;
  v.max_links = max_links;
  v.assoc_blocks = kAssocBlocksPerSM * 152;
  v.tail_blocks = 2 * 152;
  v.d_devs = reinterpret_cast<const Dev*>(dbuf + o_devs);
  for (int k = 0; k < kKinds; ++k) {
    v.tables[k].n = (int)maps[k].size();
    v.tables[k].d_map = maps[k].empty() ? nullptr : reinterpret_cast<int4*>(dbuf + o_map[k]);
  }
  v.d_ctl = reinterpret_cast<unsigned*>(dbuf + o_ctl);
  v.d_prefix = reinterpret_cast<unsigned*>(dbuf + o_prefix);
  v.d_tiles = reinterpret_cast<AssocUnit*>(dbuf + o_tiles);
  v.d_srcs = reinterpret_cast<const float* const*>(dbuf + o_srcs);
  v.host_devs = hd.data();
  v.reduce_threads = reduce_threads_for(hd.data(), n);
  enqueue_frame_view(v, st);
  const int nv = v.tables[kVerts].n;
  if (nv > 0)
    k_results_b<<<nv, 256, 0, st>>>(BatchGrid{v.d_devs, v.tables[kVerts].d_map},
                                    reinterpret_cast<const ResultDst*>(dbuf + o_dst));
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(TRK_ERR_CUDA, cudaGetErrorString(e));
  for (int k = 0; k < n; ++k) session_set_last_stream(ss[k], st);
  return TRK_OK;
}

}  // namespace trk

extern "C" {

trk_status trk_batch_create(trk_session* const* sessions, int32_t n_sessions, trk_batch** out) {
  return batch_create(sessions, n_sessions, 4 * 152, 2 * 152, out);
}

trk_status trk_batch_track_device(trk_batch* b, const float* const* d_depths, void* cuda_stream) {
  NvtxRange nv("trk_batch_track_device");
  if (!b || !d_depths) return set_error(TRK_ERR_INVALID_ARG, "trk_batch_track_device: NULL argument");
  if (!members_current(b))
    return set_error(TRK_ERR_INVALID_ARG, "trk_batch_track_device: a member was evicted since the batch was built");
  const int B = (int)b->sessions.size();
  for (int k = 0; k < B; ++k)
    if (!d_depths[k]) return set_error(TRK_ERR_INVALID_ARG, "trk_batch_track_device: NULL depth pointer");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // a ring of pinned pointer slots: a slot is rewritten only after the copy out of it has run
  const int slot = b->src_slot;
  b->src_slot = (slot + 1) % kSrcSlots;
  const float** h = b->h_srcs + (size_t)slot * B;
  cudaError_t e = cudaEventSynchronize(b->src_ev[slot]);
  if (e == cudaSuccess) {
    for (int k = 0; k < B; ++k) h[k] = d_depths[k];
    e = cudaMemcpyAsync(b->d_srcs, h, sizeof(float*) * B, cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess) e = cudaEventRecord(b->src_ev[slot], st);
  if (e == cudaSuccess) e = cudaGraphLaunch(b->graph, st);
  if (e != cudaSuccess) return set_error(TRK_ERR_CUDA, cudaGetErrorString(e));
  for (trk_session* s : b->sessions) session_set_last_stream(s, st);
  return TRK_OK;
}

trk_status trk_batch_profile(trk_batch* b, const float* const* d_depths, int32_t reps, size_t flush_bytes, float* ms) {
  if (!b || !d_depths || !ms || reps <= 0) return set_error(TRK_ERR_INVALID_ARG, "trk_batch_profile: bad arguments");
  if (!members_current(b))
    return set_error(TRK_ERR_INVALID_ARG, "trk_batch_profile: a member was evicted since the batch was built");
  const int B = (int)b->sessions.size();
  const int L = b->max_links;
  cudaStream_t st = b->cap;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  void* flush = nullptr;
  cudaError_t err = cudaEventCreate(&e0);
  if (!err) err = cudaEventCreate(&e1);
  if (!err && flush_bytes) err = cudaMalloc(&flush, flush_bytes);
  // this frame's depth (the profile starts like a frame)
  const float** h = b->h_srcs;  // slot 0; wait for any copy still reading it
  if (!err) err = cudaEventSynchronize(b->src_ev[0]);
  if (!err) {
    for (int k = 0; k < B; ++k) h[k] = d_depths[k];
    err = cudaMemcpyAsync(b->d_srcs, h, sizeof(float*) * B, cudaMemcpyHostToDevice, st);
  }
  if (!err) err = cudaEventRecord(b->src_ev[0], st);
  if (!err) err = cudaMemsetAsync(b->d_ctl, 0, sizeof(unsigned) * 3, st);
  if (!err) launch_gather_depth_b(grid_of(b, kAssoc), b->tables[kAssoc].n, b->d_srcs, b->d_tiles, b->d_ctl, st);
  double acc[TRK_STAGE_COUNT] = {0};
  int flushes = 0;
  auto timed = [&](int stage, auto&& fn) -> cudaError_t {
    if (flush) cudaMemsetAsync(flush, (flushes++) & 0xFF, flush_bytes, st);
    cudaEventRecord(e0, st);
    fn();
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) return e;
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    acc[stage] += t;
    return cudaGetLastError();
  };
  BatchGrid gj[5];
  int nj[5], nz[5] = {0, 0, 0, 0, 0};
  for (int t = 0; t < 5; ++t) {
    gj[t] = grid_of(b, (Kind)(kJtj1 + t));
    nj[t] = b->tables[kJtj1 + t].n;
  }
  for (int r = 0; r < reps && err == cudaSuccess; ++r) {
    err = timed(TRK_STAGE_SKIN, [&] { launch_skin_b(grid_of(b, kSkin), b->tables[kSkin].n, L, 0, b->d_ctl, st); });
    if (!err) err = timed(TRK_STAGE_RASTER, [&] { launch_raster_b(grid_of(b, kTris), b->tables[kTris].n, st); });
    if (!err) err = timed(TRK_STAGE_VISIBILITY, [&] { launch_visibility_b(grid_of(b, kVerts), b->tables[kVerts].n, st); });
    if (!err)
      err = timed(TRK_STAGE_ASSOCIATE, [&] {
        launch_associate_b(b->d_devs, B, b->d_tiles, b->d_ctl, b->d_prefix, b->assoc_blocks, b->tail_blocks, st);
      });
    if (!err)
      err = timed(TRK_STAGE_RESID_JTJ, [&] {
        launch_normal_equations_b(gj, nj, grid_of(b, kReduce), 0, L, b->precision, 0, -1, st, 1024);
      });
    if (!err)
      err = timed(TRK_STAGE_REDUCE, [&] {
        launch_normal_equations_b(gj, nz, grid_of(b, kReduce), b->tables[kReduce].n, L, b->precision, 0, -1, st,
                                  reduce_threads_of(b));
      });
    if (!err) err = timed(TRK_STAGE_LM_SOLVE, [&] { launch_lm_b(grid_of(b, kLm), b->tables[kLm].n, grid_of(b, kRows), 0, L, 0, st); });
    if (!err) err = timed(TRK_STAGE_LM_EVAL, [&] { launch_lm_b(grid_of(b, kLm), 0, grid_of(b, kRows), b->tables[kRows].n, L, 0, st); });
  }
  for (int r = 0; r < reps && err == cudaSuccess; ++r) {
    launch_skin_b(grid_of(b, kSkin), b->tables[kSkin].n, L, 0, b->d_ctl, st);
    launch_raster_b(grid_of(b, kTris), b->tables[kTris].n, st);
    launch_visibility_b(grid_of(b, kVerts), b->tables[kVerts].n, st);
    launch_associate_b(b->d_devs, B, b->d_tiles, b->d_ctl, b->d_prefix, b->assoc_blocks, b->tail_blocks, st);
    int cur = 0;
    err = timed(TRK_STAGE_SHAPE, [&] {
      cur = launch_shape_b(grid_of(b, kVerts), b->tables[kVerts].n, L, b->shape_sweeps, b->shape_solver, 0, -1, st);
    });
    if (!err && cur != 0)
      for (trk_session* s : b->sessions) {
        const Dev& d = session_dev(s);
        cudaMemcpyAsync(d.phi[0], d.phi[cur], sizeof(float4) * d.V, cudaMemcpyDeviceToDevice, st);
      }
  }
  cudaStreamSynchronize(st);
  if (flush) cudaFree(flush);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (err != cudaSuccess) return set_error(TRK_ERR_CUDA, cudaGetErrorString(err));
  for (int k = 0; k < TRK_STAGE_COUNT; ++k) ms[k] = (float)(acc[k] / reps);
  return TRK_OK;
}

void trk_batch_destroy(trk_batch* b) { free_batch(b); }

}  // extern "C"
