// trk_api.cu -- host side of the C ABI declared in include/trk.h: validation, derived model data
// (bind pose, prior weights, vertex-to-face lists, neighbourhoods), device allocation, the per-frame
// CUDA graph and the step-level calls.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>

#include "../../include/trk.h"
#include "trk_internal.cuh"

using namespace trk;

namespace {

thread_local std::string g_err;

trk_status fail(trk_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return fail(e_ == cudaErrorMemoryAllocation ? TRK_ERR_OOM : TRK_ERR_CUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                              \
  } while (0)

// ---- host dual quaternions in FP64 (bind pose only) ----------------------------------------------
struct HQ { double w, x, y, z; };
struct HDQ { HQ r, d; };
HQ hmul(HQ a, HQ b) {
  return {a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z, a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y,
          a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x, a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w};
}
HQ hadd(HQ a, HQ b) { return {a.w + b.w, a.x + b.x, a.y + b.y, a.z + b.z}; }
HDQ hdmul(const HDQ& a, const HDQ& b) { return {hmul(a.r, b.r), hadd(hmul(a.r, b.d), hmul(a.d, b.r))}; }

// Exact knn nearest other vertices (squared distance of the float coordinates in FP64, ties to the
// smaller index) with a uniform grid: cells are visited in rings of growing Chebyshev radius rho; once
// knn candidates are held and the k-th distance is below (rho * cell)^2, no farther cell can beat it.
void knn_grid(int V, const float* xyz, int K, std::vector<int>& nbr) {
  nbr.assign((size_t)V * 4, -1);
  if (K <= 0 || V <= 1) return;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int i = 0; i < V; ++i)
    for (int c = 0; c < 3; ++c) {
      lo[c] = std::min(lo[c], (double)xyz[3 * i + c]);
      hi[c] = std::max(hi[c], (double)xyz[3 * i + c]);
    }
  double ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
  double cell = std::max(ext / std::max(1.0, std::cbrt((double)V / 2.0)), 1e-9);
  int n[3];
  for (int c = 0; c < 3; ++c) n[c] = std::max(1, (int)std::floor((hi[c] - lo[c]) / cell) + 1);
  auto cidx = [&](int i, int c) { return std::min(n[c] - 1, (int)std::floor((xyz[3 * i + c] - lo[c]) / cell)); };
  std::vector<int> start((size_t)n[0] * n[1] * n[2] + 1, 0), list(V);
  for (int i = 0; i < V; ++i) start[((size_t)cidx(i, 2) * n[1] + cidx(i, 1)) * n[0] + cidx(i, 0) + 1]++;
  for (size_t k = 1; k < start.size(); ++k) start[k] += start[k - 1];
  std::vector<int> fill(start.begin(), start.end() - 1);
  for (int i = 0; i < V; ++i) list[fill[((size_t)cidx(i, 2) * n[1] + cidx(i, 1)) * n[0] + cidx(i, 0)]++] = i;
  const int maxr = std::max(n[0], std::max(n[1], n[2]));
  for (int i = 0; i < V; ++i) {
    double bd[4];
    int bi[4], cnt = 0;
    const int ci[3] = {cidx(i, 0), cidx(i, 1), cidx(i, 2)};
    for (int rho = 0; rho <= maxr; ++rho) {
      for (int z = ci[2] - rho; z <= ci[2] + rho; ++z) {
        if (z < 0 || z >= n[2]) continue;
        for (int y = ci[1] - rho; y <= ci[1] + rho; ++y) {
          if (y < 0 || y >= n[1]) continue;
          for (int x = ci[0] - rho; x <= ci[0] + rho; ++x) {
            if (x < 0 || x >= n[0]) continue;
            if (std::max(std::abs(x - ci[0]), std::max(std::abs(y - ci[1]), std::abs(z - ci[2]))) != rho) continue;
            const size_t q = ((size_t)z * n[1] + y) * n[0] + x;
            for (int t = start[q]; t < start[q + 1]; ++t) {
              const int j = list[t];
              if (j == i) continue;
              const double dx = (double)xyz[3 * j] - (double)xyz[3 * i];
              const double dy = (double)xyz[3 * j + 1] - (double)xyz[3 * i + 1];
              const double dz = (double)xyz[3 * j + 2] - (double)xyz[3 * i + 2];
              const double d2 = dx * dx + dy * dy + dz * dz;
              if (cnt == K && (d2 > bd[K - 1] || (d2 == bd[K - 1] && j > bi[K - 1]))) continue;
              int pos = cnt < K ? cnt++ : K - 1;
              while (pos > 0 && (bd[pos - 1] > d2 || (bd[pos - 1] == d2 && bi[pos - 1] > j))) {
                bd[pos] = bd[pos - 1];
                bi[pos] = bi[pos - 1];
                --pos;
              }
              bd[pos] = d2;
              bi[pos] = j;
            }
          }
        }
      }
      const double reach = rho * cell;
      if (cnt == K && bd[K - 1] < reach * reach * (1.0 - 1e-12)) break;
    }
    for (int k = 0; k < cnt; ++k) nbr[(size_t)i * 4 + k] = bi[k];
  }
}

}  // namespace

namespace {
// the driver's virtual memory management calls, looked up through the runtime (no link to libcuda)
struct VmmApi {
  decltype(&cuMemGetAllocationGranularity) granularity = nullptr;
  decltype(&cuMemCreate) create = nullptr;
  decltype(&cuMemRelease) release = nullptr;
  decltype(&cuMemAddressReserve) reserve = nullptr;
  decltype(&cuMemAddressFree) address_free = nullptr;
  decltype(&cuMemMap) map = nullptr;
  decltype(&cuMemUnmap) unmap = nullptr;
  decltype(&cuMemSetAccess) set_access = nullptr;
  bool ok = false;
};
std::mutex g_vmm_mu;
VmmApi g_vmm;
bool g_vmm_loaded = false;
std::atomic<size_t> g_vmm_held{0};

template <typename F>
bool entry(const char* name, F* fn) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q{};
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !p)
    return false;
  *fn = reinterpret_cast<F>(p);
  return true;
}

const VmmApi& vmm() {
  std::lock_guard<std::mutex> lk(g_vmm_mu);
  if (!g_vmm_loaded) {
    g_vmm_loaded = true;
    VmmApi a;
    a.ok = entry("cuMemGetAllocationGranularity", &a.granularity) && entry("cuMemCreate", &a.create) &&
           entry("cuMemRelease", &a.release) && entry("cuMemAddressReserve", &a.reserve) &&
           entry("cuMemAddressFree", &a.address_free) && entry("cuMemMap", &a.map) &&
           entry("cuMemUnmap", &a.unmap) && entry("cuMemSetAccess", &a.set_access);
    g_vmm = a;
  }
  return g_vmm;
}

CUmemAllocationProp device_prop(int dev) {
  CUmemAllocationProp prop{};
  prop.type = CU_MEM_ALLOCATION_TYPE_PINNED;
  prop.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
  prop.location.id = dev;
  return prop;
}
}  // namespace

size_t trk::vmm_granularity() {
  const VmmApi& a = vmm();
  int dev = 0;
  if (!a.ok || cudaGetDevice(&dev) != cudaSuccess) return 0;
  const CUmemAllocationProp prop = device_prop(dev);
  size_t g = 0;
  if (a.granularity(&g, &prop, CU_MEM_ALLOC_GRANULARITY_MINIMUM) != CUDA_SUCCESS) return 0;
  return g;
}

cudaError_t trk::vmm_alloc(size_t bytes, VmmBlock* out) {
  const VmmApi& a = vmm();
  if (!a.ok) return cudaErrorNotSupported;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const size_t g = vmm_granularity();
  if (!g) return cudaErrorNotSupported;
  const size_t size = (std::max<size_t>(bytes, 1) + g - 1) / g * g;
  const CUmemAllocationProp prop = device_prop(dev);
  CUmemGenericAllocationHandle h = 0;
  if (a.create(&h, size, &prop, 0) != CUDA_SUCCESS) return cudaErrorMemoryAllocation;
  CUdeviceptr ptr = 0;
  if (a.reserve(&ptr, size, g, 0, 0) != CUDA_SUCCESS) {
    a.release(h);
    return cudaErrorMemoryAllocation;
  }
  CUmemAccessDesc acc{};
  acc.location = prop.location;
  acc.flags = CU_MEM_ACCESS_FLAGS_PROT_READWRITE;
  if (a.map(ptr, size, 0, h, 0) != CUDA_SUCCESS) {
    a.address_free(ptr, size);
    a.release(h);
    return cudaErrorMemoryAllocation;
  }
  if (a.set_access(ptr, size, &acc, 1) != CUDA_SUCCESS) {
    a.unmap(ptr, size);
    a.address_free(ptr, size);
    a.release(h);
    return cudaErrorMemoryAllocation;
  }
  out->ptr = reinterpret_cast<void*>(ptr);
  out->size = size;
  out->handle = (unsigned long long)h;
  g_vmm_held += size;
  return cudaSuccess;
}

void trk::vmm_free(VmmBlock* b) {
  if (!b || !b->ptr) return;
  const VmmApi& a = vmm();
  const CUdeviceptr ptr = reinterpret_cast<CUdeviceptr>(b->ptr);
  a.unmap(ptr, b->size);
  a.address_free(ptr, b->size);
  a.release((CUmemGenericAllocationHandle)b->handle);
  g_vmm_held -= b->size;
  *b = VmmBlock{};
}

size_t trk::vmm_bytes_held() { return g_vmm_held.load(); }

int trk::set_error_code(int st, const char* msg) {
  g_err = msg ? msg : "";
  return st;
}

// Model data a session keeps on the host, so that its device state can be freed (evicted) and made
// again (restored) without the caller's arrays.
struct HostModel {
  LinkTable lt{};
  std::vector<float4> v0, bw;
  std::vector<uchar4> bidx;
  std::vector<int4> tris, nb;
  std::vector<int> csr_off, csr_face, adj_off, adj;
  std::vector<double> prior2;
};

struct trk_session {
  Dev d{};
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t last_stream = nullptr;
  cudaGraphExec_t graph = nullptr;       // a frame with the shape iterations
  cudaGraphExec_t graph_pose = nullptr;  // a frame of pose iterations only (shape-match after frame 0, smooth-bind)
  int frames_done = 0;                   // frames since the last trk_set_pose
  trk_params prm{};
  HostModel hm;
  bool resident = false;    // the device state exists
  unsigned generation = 0;  // changes whenever the device state is made or freed
  void* arena = nullptr;    // one device block (vmm_alloc) holding every device buffer of the session
  VmmBlock block;           // the block behind the arena
  size_t carved = 0;        // bytes of the arena handed out so far (or, without an arena, counted)
  size_t device_bytes = 0;  // size of the arena: the carved bytes rounded up to the allocation granularity
  // the tracking state while the session is evicted: Theta, lambda, Phi
  std::vector<double> ev_theta;
  double ev_lam = 0.0;
  std::vector<float4> ev_phi;
  double* h_pinned = nullptr;  // pinned staging for results
  float4* h_phi = nullptr;     // pinned staging for the offsets of a result [V]
  float* d_render = nullptr;
};

namespace {

trk_status materialize(trk_session* s);
trk_status evict(trk_session* s);

// Hands out the next piece of the session's arena (256-byte aligned).  Without an arena it only
// counts, and the pointer is NULL: carve_all() run that way gives the arena's size.
template <typename T>
void carve(trk_session* s, T** p, size_t count) {
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  s->carved = (s->carved + 255) & ~size_t(255);
  *p = s->arena ? reinterpret_cast<T*>(static_cast<char*>(s->arena) + s->carved) : nullptr;
  s->carved += bytes;
}

#define TRY(x)                         \
  do {                                 \
    trk_status st_ = (x);              \
    if (st_ != TRK_OK) return st_;     \
  } while (0)

// Calls that run kernels or read device buffers need the device state.
#define NEED_RESIDENT(s)                                                                              \
  do {                                                                                              \
    if (!(s)->resident) return fail(TRK_ERR_INVALID_ARG, "the session is evicted (trk_session_restore)"); \
  } while (0)

trk_status validate(const trk_mesh* m, const trk_skeleton* k, const trk_intrinsics* c, const trk_params* p) {
  if (!m || !k || !c || !p) return fail(TRK_ERR_INVALID_ARG, "NULL argument");
  if (k->n_links <= 0) return fail(TRK_ERR_INVALID_ARG, "n_links must be positive");
  if (k->n_links > TRK_MAX_LINKS) return fail(TRK_ERR_NO_CAPACITY, "n_links %d > %d", k->n_links, TRK_MAX_LINKS);
  if (m->n_verts <= 0 || m->n_tris < 0) return fail(TRK_ERR_INVALID_ARG, "bad mesh sizes");
  if (!m->verts || !m->bone_idx || !m->bone_w || (m->n_tris && !m->tris)) return fail(TRK_ERR_INVALID_ARG, "NULL mesh array");
  if (!k->parent || !k->type || !k->axis || !k->offset_dq || !k->prior_mask)
    return fail(TRK_ERR_INVALID_ARG, "NULL skeleton array");
  if (c->width <= 0 || c->height <= 0 || !(c->fx > 0) || !(c->fy > 0) || !std::isfinite(c->cx) || !std::isfinite(c->cy))
    return fail(TRK_ERR_INVALID_ARG, "bad intrinsics");
  if ((long long)c->width * c->height > (1ll << 28)) return fail(TRK_ERR_NO_CAPACITY, "image too large");
  if (p->precision != TRK_PRECISION_FP32 && p->precision != TRK_PRECISION_BF16X3 &&
      p->precision != TRK_PRECISION_TF32X3)
    return fail(TRK_ERR_INVALID_ARG, "precision %d not supported", p->precision);
  if (p->shape_solver != 0 && p->shape_solver != 1)
    return fail(TRK_ERR_INVALID_ARG, "shape_solver %d not supported", p->shape_solver);
  if (p->mode != TRK_MODE_TRACK && p->mode != TRK_MODE_SHAPE_MATCH && p->mode != TRK_MODE_SMOOTH_BIND)
    return fail(TRK_ERR_INVALID_ARG, "mode %d not supported", p->mode);
  if (p->association != 0 && p->association != 1)
    return fail(TRK_ERR_INVALID_ARG, "association %d not supported", p->association);
  if (p->jtj_group != 0 && p->jtj_group != 1 && p->jtj_group != 2 && p->jtj_group != 4)
    return fail(TRK_ERR_INVALID_ARG, "jtj_group %d not supported", p->jtj_group);
  if (p->pose_iters < 0 || p->shape_iters < 0 || p->shape_sweeps < 1 || p->knn < 0 || p->knn > 4 ||
      p->window_half_px < 0 || !(p->cutoff_m > 0) || !(p->lambda_k0 > 0) || p->lambda_s < 0 || p->lambda_phi < 0 ||
      p->lambda_N < 0 || p->lambda_w < 0 || !(p->z_near_m > 0) || !(p->eps_vis_m >= 0))
    return fail(TRK_ERR_INVALID_ARG, "bad params");
  const int L = k->n_links;
  for (int j = 0; j < L; ++j) {
    if (k->parent[j] >= j || k->parent[j] < -1) return fail(TRK_ERR_INVALID_ARG, "parent[%d] must be in [-1, %d)", j, j);
    if (k->type[j] != 0 && k->type[j] != 1) return fail(TRK_ERR_INVALID_ARG, "type[%d]", j);
    const float* a = k->axis + 3 * j;
    const double an = std::sqrt((double)a[0] * a[0] + (double)a[1] * a[1] + (double)a[2] * a[2]);
    if (!(an > 0.5 && an < 2.0)) return fail(TRK_ERR_INVALID_ARG, "axis[%d] not unit", j);
    const float* o = k->offset_dq + 8 * j;
    double nr = 0, od = 0;
    for (int q = 0; q < 4; ++q) { nr += (double)o[q] * o[q]; od += (double)o[q] * o[4 + q]; }
    if (std::fabs(nr - 1.0) > 1e-5 || std::fabs(od) > 1e-5) return fail(TRK_ERR_INVALID_ARG, "offset_dq[%d] not unit", j);
    if (!std::isfinite(k->prior_mask[j])) return fail(TRK_ERR_INVALID_ARG, "prior_mask[%d]", j);
  }
  for (long long t = 0; t < 3ll * m->n_tris; ++t)
    if (m->tris[t] < 0 || m->tris[t] >= m->n_verts) return fail(TRK_ERR_INVALID_ARG, "tris[%lld] out of range", t);
  for (int i = 0; i < m->n_verts; ++i) {
    double sw = 0;
    for (int q = 0; q < 4; ++q) {
      const float w = m->bone_w[4 * i + q];
      if (!(w >= 0) || m->bone_idx[4 * i + q] >= L) return fail(TRK_ERR_INVALID_ARG, "bone slot %d of vertex %d", q, i);
      sw += w;
    }
    if (std::fabs(sw - 1.0) > 1e-4) return fail(TRK_ERR_INVALID_ARG, "weights of vertex %d sum to %g", i, sw);
    for (int c2 = 0; c2 < 3; ++c2)
      if (!std::isfinite(m->verts[3 * i + c2])) return fail(TRK_ERR_NUMERIC, "vertex %d not finite", i);
  }
  return TRK_OK;
}

// Records the whole frame (pose iterations, then shape iterations) on st.
void enqueue_frame(trk_session* s, cudaStream_t st, bool with_shape) {
  const Dev& d = s->d;
  const int P = s->prm.pose_iters, S = with_shape ? s->prm.shape_iters : 0;
  int cur = 0;
  // a frame without shape iterations reports NaN for their energies (all-ones bytes are a NaN)
  if (!with_shape && s->prm.shape_iters > 0) cudaMemsetAsync(d.energy + P, 0xFF, sizeof(double) * s->prm.shape_iters, st);
  for (int it = 0; it < P; ++it) {
    NvtxRange nv("pose iteration");
    launch_skin(d, cur, st);
    launch_raster(d, st);
    launch_visibility(d, st);
    launch_associate(d, st);
    launch_normal_equations(d, cur, it, st);
    launch_lm(d, cur, st);
  }
  for (int it = 0; it < S; ++it) {
    NvtxRange nv("shape iteration");
    launch_skin(d, cur, st);
    launch_raster(d, st);
    launch_visibility(d, st);
    launch_associate(d, st);
    cur = launch_shape(d, cur, P + it, st);
  }
  if (cur != 0) cudaMemcpyAsync(d.phi[0], d.phi[cur], sizeof(float4) * d.V, cudaMemcpyDeviceToDevice, st);
}

// Whether the next frame runs the shape iterations: always in tracking mode, on the first frame after
// trk_set_pose in shape-match mode, never in smooth-bind mode.
bool next_frame_with_shape(const trk_session* s) {
  return s->prm.mode == TRK_MODE_TRACK || (s->prm.mode == TRK_MODE_SHAPE_MATCH && s->frames_done == 0);
}

// The frame graph for the next frame (captured on first use).
trk_status frame_graph(trk_session* s, cudaGraphExec_t* out) {
  const bool with_shape = next_frame_with_shape(s);
  cudaGraphExec_t& ge = with_shape ? s->graph : s->graph_pose;
  if (!ge) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    enqueue_frame(s, s->stream, with_shape);
    CK(cudaStreamEndCapture(s->stream, &g));
    cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    CK(e);
  }
  *out = ge;
  return TRK_OK;
}

trk_status fetch_result(trk_session* s, cudaStream_t st, trk_result* out) {
  if (!out) return TRK_OK;
  const Dev& d = s->d;
  const int ne = s->prm.pose_iters + s->prm.shape_iters;
  double* h = s->h_pinned;  // [L] theta, [ne] energy, [1] stats
  CK(cudaMemcpyAsync(h, d.theta, sizeof(double) * d.L, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h + d.L, d.energy, sizeof(double) * ne, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h + d.L + ne, d.stats, sizeof(int) * 4, cudaMemcpyDeviceToHost, st));
  const float4* phi = s->h_phi;
  if (out->offsets) CK(cudaMemcpyAsync(s->h_phi, d.phi[0], sizeof(float4) * d.V, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (out->theta) std::memcpy(out->theta, h, sizeof(double) * d.L);
  if (out->energy) std::memcpy(out->energy, h + d.L, sizeof(double) * ne);
  int stats[4];
  std::memcpy(stats, h + d.L + ne, sizeof(stats));
  out->n_assoc_px = stats[0];
  out->n_assoc_verts = stats[1];
  if (stats[3]) return fail(TRK_ERR_TIMEOUT, "a tensor-core completion wait ran out; results are not valid");
  if (out->offsets)
    for (int i = 0; i < d.V; ++i) {
      out->offsets[3 * i] = phi[i].x;
      out->offsets[3 * i + 1] = phi[i].y;
      out->offsets[3 * i + 2] = phi[i].z;
    }
  return TRK_OK;
}

trk_status sync_check(trk_session* s) {
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s->stream));
  return TRK_OK;
}

}  // namespace

// ---- helpers of the frame server (server.cu) --------------------------------------------------
namespace trk {
size_t session_device_bytes(const trk_session* s) { return s->device_bytes; }
bool session_resident(const trk_session* s) { return s->resident; }
unsigned session_generation(const trk_session* s) { return s->generation; }
trk_status session_evict(trk_session* s) { return evict(s); }
trk_status session_restore(trk_session* s) { return materialize(s); }
const Dev& session_dev(const trk_session* s) { return s->d; }
const trk_params& session_params(const trk_session* s) { return s->prm; }
void session_set_last_stream(trk_session* s, cudaStream_t st) { s->last_stream = st; }
// The owner of stream st has waited for it and is about to destroy it: the session's last frame there is done.
void session_forget_stream(trk_session* s, cudaStream_t st) {
  if (s->last_stream == st) s->last_stream = nullptr;
}
int session_device(const trk_session* s) { return s->device; }
void session_result_sizes(const trk_session* s, int* n_links, int* n_verts, int* n_energy) {
  *n_links = s->d.L;
  *n_verts = s->d.V;
  *n_energy = s->prm.pose_iters + s->prm.shape_iters;
}
// H2D of the frame's depth and the frame graph, on the session's stream
trk_status session_enqueue_frame(trk_session* s, const float* host_depth, cudaStream_t* stream_out) {
  cudaGraphExec_t ge;
  TRY(frame_graph(s, &ge));
  CK(cudaMemcpyAsync(const_cast<float*>(s->d.depth), host_depth, sizeof(float) * s->d.cam.W * s->d.cam.H,
                     cudaMemcpyHostToDevice, s->stream));
  launch_tiles(s->d, s->d.depth, s->stream);  // the frame's occupied tiles (the graph's association reads them)
  CK(cudaGraphLaunch(ge, s->stream));
  ++s->frames_done;
  s->last_stream = s->stream;
  *stream_out = s->stream;
  return TRK_OK;
}
// D2H of the frame's results into (pinned) host buffers, on the session's stream
trk_status session_enqueue_results(trk_session* s, double* theta, float* phi4, double* energy, int* stats) {
  const Dev& d = s->d;
  const int ne = s->prm.pose_iters + s->prm.shape_iters;
  CK(cudaMemcpyAsync(theta, d.theta, sizeof(double) * d.L, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(phi4, d.phi[0], sizeof(float4) * d.V, cudaMemcpyDeviceToHost, s->stream));
  if (ne > 0) CK(cudaMemcpyAsync(energy, d.energy, sizeof(double) * ne, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(stats, d.stats, sizeof(int) * 4, cudaMemcpyDeviceToHost, s->stream));
  return TRK_OK;
}
}  // namespace trk

extern "C" {

const char* trk_last_error(void) { return g_err.c_str(); }

void trk_destroy(trk_session* s) {
  if (!s) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(s->device);
  if (s->last_stream && s->last_stream != s->stream) cudaStreamSynchronize(s->last_stream);
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->graph) cudaGraphExecDestroy(s->graph);
  if (s->graph_pose) cudaGraphExecDestroy(s->graph_pose);
  if (s->arena) vmm_free(&s->block);  // the streams above are idle
  if (s->h_pinned) cudaFreeHost(s->h_pinned);
  if (s->h_phi) cudaFreeHost(s->h_phi);
  if (s->stream) cudaStreamDestroy(s->stream);
  cudaSetDevice(cur);
  cudaGetLastError();  // the calls above are not checked: leave no error behind for the caller's next call
  delete s;
}

}  // extern "C"

namespace {

// Every device buffer of a session, carved from its arena in a fixed order (or only counted).
void carve_all(trk_session* s) {
  Dev& d = s->d;
  const trk_params& prm = s->prm;
  const int L = d.L, V = d.V, F = d.F, NP = d.NP;
  const size_t npx = (size_t)d.cam.W * d.cam.H;
  s->carved = 0;
  LinkTable* dlt;
  float4 *dv0, *dbw;
  uchar4* dbidx;
  int4 *dtris, *dnb;
  int *dcsr_off, *dcsr_face, *dadj_off, *dadj;
  double* dprior;
  float* ddepth;
  carve(s, &dlt, 1);
  carve(s, &dv0, V); carve(s, &dbw, V); carve(s, &dbidx, V);
  carve(s, &dtris, F); carve(s, &dnb, V);
  carve(s, &dcsr_off, V + 1); carve(s, &dcsr_face, (size_t)3 * F);
  carve(s, &dprior, L);
  carve(s, &d.phi[0], V); carve(s, &d.phi[1], V);
  carve(s, &d.theta, L); carve(s, &d.lam, 1);
  carve(s, &d.energy, std::max(1, prm.pose_iters + prm.shape_iters));
  carve(s, &d.Hd, L); carve(s, &d.xi, (size_t)8 * L);
  carve(s, &d.theta_c, (size_t)kCandidates * L); carve(s, &d.Hd_c, (size_t)kCandidates * L);
  carve(s, &d.xi_c, (size_t)kCandidates * L * 8); carve(s, &d.lm_trials, 8);
  carve(s, &d.lm_ok, 2 * kCandidates);
  carve(s, &d.v, V); carve(s, &d.n, V); carve(s, &d.fn, F); carve(s, &d.rec, V);
  carve(s, &d.head, npx); carve(s, &d.zbuf, npx); carve(s, &d.corr, npx);
  carve(s, &d.pixrec, npx); carve(s, &d.queue, npx); carve(s, &d.qctl, 4);
  carve(s, &d.units, (size_t)kUnitsPerTile * ((d.cam.W + 15) / 16) * ((d.cam.H + 15) / 16));
  carve(s, &d.acc, V); carve(s, &d.vispix, V); carve(s, &d.rg, V); carve(s, &d.phi0, V);
  carve(s, &dadj_off, V + 1); carve(s, &dadj, s->hm.adj.size());
  d.cg_x = d.cg_r = d.cg_z = d.cg_p = d.cg_ap = nullptr;
  if (prm.shape_solver == 1) {
    carve(s, &d.cg_x, V); carve(s, &d.cg_r, V); carve(s, &d.cg_z, V);
    carve(s, &d.cg_p, V); carve(s, &d.cg_ap, V);
  }
  carve(s, &d.cg, 4);
  carve(s, &ddepth, npx);
  carve(s, &s->d_render, npx);
  carve(s, &d.partial, (size_t)d.nblk_rows * NP * NP);
  carve(s, &d.jtj_rows, (size_t)d.nblk_rows);
  carve(s, &d.arec, (size_t)d.nblk_jtj * 256 * 4);
  carve(s, &d.A, (size_t)NP * NP);
  carve(s, &d.epart, (size_t)std::max(d.nblk_v, 1) * 8);
  carve(s, &d.counter, 4);
  carve(s, &d.stats, 4);
  d.links = dlt; d.v0 = dv0; d.bw = dbw; d.bidx = dbidx; d.tris = dtris; d.nbr = dnb;
  d.csr_off = dcsr_off; d.csr_face = dcsr_face; d.prior2 = dprior;
  d.depth = ddepth;
  d.adj_off = dadj_off;
  d.adj = dadj;
}

// Makes the device state: one arena (a device block of vmm_alloc), the model data uploaded from the
// host copy, the work buffers initialised and the tracking state (Theta, lambda, Phi) restored.
trk_status materialize(trk_session* s) {
  if (s->resident) return TRK_OK;
  carve_all(s);  // sizing pass (no arena yet)
  const size_t bytes = s->carved;
  cudaError_t e = vmm_alloc(bytes, &s->block);
  if (e != cudaSuccess)
    return fail(e == cudaErrorMemoryAllocation ? TRK_ERR_OOM : TRK_ERR_CUDA, "device state of %zu bytes: %s", bytes,
                cudaGetErrorString(e));
  s->arena = s->block.ptr;
  struct Undo {
    trk_session* s;
    bool armed = true;
    ~Undo() {
      if (!armed) return;
      cudaStreamSynchronize(s->stream);
      vmm_free(&s->block);
      s->arena = nullptr;
      carve_all(s);
    }
  } undo{s};
  if (reinterpret_cast<uintptr_t>(s->arena) % 256 != 0)
    return fail(TRK_ERR_CUDA, "device state allocation not 256-byte aligned");
  s->device_bytes = s->block.size;
  carve_all(s);
  Dev& d = s->d;
  const HostModel& hm = s->hm;
  const int L = d.L, V = d.V, F = d.F;
  const size_t npx = (size_t)d.cam.W * d.cam.H;
  const int ne = std::max(1, s->prm.pose_iters + s->prm.shape_iters);
  cudaStream_t st = s->stream;
  CK(cudaMemcpyAsync(const_cast<LinkTable*>(d.links), &hm.lt, sizeof(LinkTable), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(const_cast<float4*>(d.v0), hm.v0.data(), sizeof(float4) * V, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(const_cast<float4*>(d.bw), hm.bw.data(), sizeof(float4) * V, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(const_cast<uchar4*>(d.bidx), hm.bidx.data(), sizeof(uchar4) * V, cudaMemcpyHostToDevice, st));
  if (F) CK(cudaMemcpyAsync(const_cast<int4*>(d.tris), hm.tris.data(), sizeof(int4) * F, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(const_cast<int4*>(d.nbr), hm.nb.data(), sizeof(int4) * V, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(const_cast<int*>(d.csr_off), hm.csr_off.data(), sizeof(int) * (V + 1), cudaMemcpyHostToDevice, st));
  if (F) CK(cudaMemcpyAsync(const_cast<int*>(d.csr_face), hm.csr_face.data(), sizeof(int) * 3 * F, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(const_cast<double*>(d.prior2), hm.prior2.data(), sizeof(double) * L, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(const_cast<int*>(d.adj_off), hm.adj_off.data(), sizeof(int) * (V + 1), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(const_cast<int*>(d.adj), hm.adj.data(), sizeof(int) * hm.adj.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(d.cg, 0, sizeof(double) * 4, st));
  CK(cudaMemsetAsync(d.counter, 0, sizeof(unsigned) * 4, st));
  CK(cudaMemsetAsync(d.qctl, 0, sizeof(unsigned) * 4, st));
  CK(cudaMemsetAsync(d.stats, 0, sizeof(int) * 4, st));
  CK(cudaMemsetAsync(d.energy, 0, sizeof(double) * ne, st));
  CK(cudaMemsetAsync(d.lm_trials, 0, sizeof(double) * 8, st));
  CK(cudaMemsetAsync(const_cast<float*>(d.depth), 0, sizeof(float) * npx, st));
  // the tracking state
  CK(cudaMemcpyAsync(d.theta, s->ev_theta.data(), sizeof(double) * L, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d.lam, &s->ev_lam, sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d.phi[0], s->ev_phi.data(), sizeof(float4) * V, cudaMemcpyHostToDevice, st));
  launch_fk(d, st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  undo.armed = false;
  s->resident = true;
  s->last_stream = nullptr;
  ++s->generation;
  return TRK_OK;
}

// Frees the device state after saving the tracking state on the host (frame graphs go with it).
trk_status evict(trk_session* s) {
  if (!s->resident) return TRK_OK;
  const Dev& d = s->d;
  if (s->last_stream && s->last_stream != s->stream) CK(cudaStreamSynchronize(s->last_stream));
  CK(cudaMemcpyAsync(s->ev_theta.data(), d.theta, sizeof(double) * d.L, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(&s->ev_lam, d.lam, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaMemcpyAsync(s->ev_phi.data(), d.phi[0], sizeof(float4) * d.V, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  if (s->graph) cudaGraphExecDestroy(s->graph);
  if (s->graph_pose) cudaGraphExecDestroy(s->graph_pose);
  s->graph = s->graph_pose = nullptr;
  vmm_free(&s->block);  // the memory is back on the device when the eviction returns
  s->arena = nullptr;
  carve_all(s);  // every device pointer back to NULL
  s->resident = false;
  s->last_stream = nullptr;
  ++s->generation;
  return TRK_OK;
}

trk_status create_session(const trk_mesh* mesh, const trk_skeleton* sk, const trk_intrinsics* cam,
                          const trk_params* prm, bool resident, trk_session** out) {
  g_err.clear();
  if (!out) return fail(TRK_ERR_INVALID_ARG, "out is NULL");
  TRY(validate(mesh, sk, cam, prm));
  cudaGetLastError();  // an error an earlier unchecked call left on this thread is not this call's
  trk_session* s = new trk_session();
  struct Guard {
    trk_session*& s;
    ~Guard() { if (s) trk_destroy(s); }
  } guard{s};
  CK(cudaGetDevice(&s->device));
  ensure_configured();
  CK(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
  s->prm = *prm;
  const int L = sk->n_links, V = mesh->n_verts, F = mesh->n_tris, W = cam->width, H = cam->height;
  Dev& d = s->d;
  d.V = V; d.F = F; d.L = L; d.NP = L + 1;
  d.pose_iters = prm->pose_iters; d.shape_iters = prm->shape_iters; d.shape_sweeps = prm->shape_sweeps;
  d.knn = prm->knn;
  d.precision = prm->precision;
  d.shape_solver = prm->shape_solver;
  d.association = prm->association;
  d.lambda_phi = prm->lambda_phi; d.lambda_N = prm->lambda_N; d.lambda_w = prm->lambda_w;
  d.cam.W = W; d.cam.H = H; d.cam.fx = cam->fx; d.cam.fy = cam->fy; d.cam.cx = cam->cx; d.cam.cy = cam->cy;
  d.cam.z_near = prm->z_near_m; d.cam.eps_vis = prm->eps_vis_m; d.cam.tau = prm->cutoff_m; d.cam.R = prm->window_half_px;
  {  // ring bound: a vertex whose rounded pixel is >= r+1 away projects >= r+1/2 px away, i.e. at an angle
     // whose distance from p is >= d (r+1/2) / (f sqrt(1 + c_max^2)), c_max = largest |x/z| in the image
    const double cmx = std::max(cam->cx + 0.5, W - 0.5 - cam->cx) / cam->fx;
    const double cmy = std::max(cam->cy + 0.5, H - 0.5 - cam->cy) / cam->fy;
    const double kx = 1.0 / (cam->fx * std::sqrt(1.0 + cmx * cmx)), ky = 1.0 / (cam->fy * std::sqrt(1.0 + cmy * cmy));
    d.cam.kappa = (float)(std::min(kx, ky) * (1.0 - 1e-4));
  }
  // ---- session-local frame: origin at the bind-pose centroid of the template -----------------------
  double org[3] = {0, 0, 0};
  for (int i = 0; i < V; ++i)
    for (int c = 0; c < 3; ++c) org[c] += mesh->verts[3 * i + c];
  for (int c = 0; c < 3; ++c) org[c] = (double)(float)(org[c] / V);
  d.cam.ox = (float)org[0]; d.cam.oy = (float)org[1]; d.cam.oz = (float)org[2];
  d.cam.inv_fx = 1.0 / (double)cam->fx;
  d.cam.inv_fy = 1.0 / (double)cam->fy;
  const HDQ pre{{1, 0, 0, 0}, {0, -0.5 * org[0], -0.5 * org[1], -0.5 * org[2]}};  // T(-c)
  // ---- link table: normalised axes, offsets, conj(bind) from FK at Theta = 0 in FP64 ----------------
  LinkTable lt{};
  lt.L = L;
  lt.max_depth = 0;
  for (int j = 0; j < L; ++j) {
    lt.depth[j] = sk->parent[j] < 0 ? 0 : lt.depth[sk->parent[j]] + 1;
    lt.max_depth = std::max(lt.max_depth, lt.depth[j]);
  }
  {  // chains of single-child links (parents precede their children), grouped in rounds
    std::vector<int> nchild(L, 0), only_child(L, -1), chain_of(L, -1), round_of_chain;
    for (int j = 0; j < L; ++j)
      if (sk->parent[j] >= 0) {
        ++nchild[sk->parent[j]];
        only_child[sk->parent[j]] = j;
      }
    std::vector<std::vector<int>> chains;
    for (int h = 0; h < L; ++h) {
      const int p = sk->parent[h];
      if (p >= 0 && nchild[p] == 1) continue;  // continues its parent's chain
      const int c = (int)chains.size();
      chains.emplace_back();
      round_of_chain.push_back(p < 0 ? 0 : round_of_chain[chain_of[p]] + 1);
      for (int j = h;; j = only_child[j]) {
        chains[c].push_back(j);
        chain_of[j] = c;
        if (nchild[j] != 1) break;
      }
    }
    const int nc = (int)chains.size();
    int nr = 0;
    for (int c = 0; c < nc; ++c) nr = std::max(nr, round_of_chain[c] + 1);
    lt.n_chains = nc;
    lt.n_rounds = nr;
    int t = 0, k = 0;
    for (int r = 0; r < nr; ++r) {
      lt.round_start[r] = k;
      for (int c = 0; c < nc; ++c) {
        if (round_of_chain[c] != r) continue;
        lt.chain_start[k++] = t;
        for (int j : chains[c]) lt.chain[t++] = j;
      }
    }
    lt.round_start[nr] = k;
    lt.chain_start[k] = t;
  }
  lt.pre.r = make_float4(1.f, 0.f, 0.f, 0.f);
  lt.pre.d = make_float4(0.f, (float)pre.d.x, (float)pre.d.y, (float)pre.d.z);
  std::vector<HDQ> bind(L);
  for (int j = 0; j < L; ++j) {
    lt.parent[j] = sk->parent[j];
    lt.type[j] = sk->type[j];
    const float* a = sk->axis + 3 * j;
    const double an = std::sqrt((double)a[0] * a[0] + (double)a[1] * a[1] + (double)a[2] * a[2]);
    for (int c = 0; c < 3; ++c) lt.axis[j][c] = (float)(a[c] / an);
    const float* o = sk->offset_dq + 8 * j;
    lt.off[j].r = make_float4(o[0], o[1], o[2], o[3]);
    lt.off[j].d = make_float4(o[4], o[5], o[6], o[7]);
    HDQ off{{o[0], o[1], o[2], o[3]}, {o[4], o[5], o[6], o[7]}};
    HDQ par = sk->parent[j] < 0 ? pre : bind[sk->parent[j]];
    bind[j] = hdmul(par, off);  // the joint is the identity at theta = 0
    lt.bindc[j].r = make_float4((float)bind[j].r.w, (float)-bind[j].r.x, (float)-bind[j].r.y, (float)-bind[j].r.z);
    lt.bindc[j].d = make_float4((float)bind[j].d.w, (float)-bind[j].d.x, (float)-bind[j].d.y, (float)-bind[j].d.z);
  }
  // ---- prior weights: (lambda_s S_kk)^2, S_kk = mask_k n_k / |V| --------------------------------------
  std::vector<double> prior2(L, 0.0);
  {
    std::vector<int> stamp(L, -1);
    std::vector<double> cnt(L, 0.0);
    for (int i = 0; i < V; ++i)
      for (int q = 0; q < 4; ++q) {
        if (!(mesh->bone_w[4 * i + q] > 0)) continue;
        for (int k = mesh->bone_idx[4 * i + q]; k >= 0; k = sk->parent[k])
          if (stamp[k] != i) { stamp[k] = i; cnt[k] += 1.0; }
      }
    for (int k = 0; k < L; ++k) {
      const double S = (double)sk->prior_mask[k] * cnt[k] / (double)V;
      prior2[k] = ((double)prm->lambda_s * S) * ((double)prm->lambda_s * S);
    }
  }
  // ---- vertex -> face lists (faces in ascending order) ---------------------------------------------
  std::vector<int> csr_off(V + 1, 0), csr_face((size_t)3 * F);
  for (long long t = 0; t < 3ll * F; ++t) csr_off[mesh->tris[t] + 1]++;
  for (int i = 0; i < V; ++i) csr_off[i + 1] += csr_off[i];
  {
    std::vector<int> fill(csr_off.begin(), csr_off.end() - 1);
    for (int f = 0; f < F; ++f)
      for (int c = 0; c < 3; ++c) csr_face[fill[mesh->tris[3 * f + c]]++] = f;
  }
  std::vector<int> nbr;
  knn_grid(V, mesh->verts, prm->knn, nbr);
  // neighbourhood edges in both directions (the coupled shape step), each list sorted
  std::vector<int> adj_off(V + 1, 0), adj;
  for (int i = 0; i < V; ++i)
    for (int k = 0; k < 4; ++k) {
      const int q = nbr[4 * (size_t)i + k];
      if (q < 0) continue;
      adj_off[i + 1]++;
      adj_off[q + 1]++;
    }
  for (int i = 0; i < V; ++i) adj_off[i + 1] += adj_off[i];
  adj.resize(std::max(adj_off[V], 1));
  {
    std::vector<int> fill(adj_off.begin(), adj_off.end() - 1);
    for (int i = 0; i < V; ++i)
      for (int k = 0; k < 4; ++k) {
        const int q = nbr[4 * (size_t)i + k];
        if (q < 0) continue;
        adj[fill[i]++] = q;
        adj[fill[q]++] = i;
      }
    for (int i = 0; i < V; ++i) std::sort(adj.begin() + adj_off[i], adj.begin() + adj_off[i + 1]);
  }
  // ---- host staging of per-vertex / per-face arrays -----------------------------------------------
  std::vector<float4> v0(V), bw(V);
  std::vector<uchar4> bidx(V);
  std::vector<int4> tris(F), nb(V);
  for (int i = 0; i < V; ++i) {
    v0[i] = make_float4((float)(mesh->verts[3 * i] - org[0]), (float)(mesh->verts[3 * i + 1] - org[1]),
                        (float)(mesh->verts[3 * i + 2] - org[2]), 0.f);
    bw[i] = make_float4(mesh->bone_w[4 * i], mesh->bone_w[4 * i + 1], mesh->bone_w[4 * i + 2], mesh->bone_w[4 * i + 3]);
    bidx[i] = make_uchar4(mesh->bone_idx[4 * i], mesh->bone_idx[4 * i + 1], mesh->bone_idx[4 * i + 2], mesh->bone_idx[4 * i + 3]);
    nb[i] = make_int4(nbr[4 * i], nbr[4 * i + 1], nbr[4 * i + 2], nbr[4 * i + 3]);
  }
  for (int f = 0; f < F; ++f) tris[f] = make_int4(mesh->tris[3 * f], mesh->tris[3 * f + 1], mesh->tris[3 * f + 2], 0);
  HostModel& hm = s->hm;
  hm.lt = lt;
  hm.v0 = std::move(v0); hm.bw = std::move(bw); hm.bidx = std::move(bidx);
  hm.tris = std::move(tris); hm.nb = std::move(nb);
  hm.csr_off = std::move(csr_off); hm.csr_face = std::move(csr_face);
  hm.adj_off = std::move(adj_off); hm.adj = std::move(adj);
  hm.prior2 = std::move(prior2);
  // ---- [J r] block grouping ---------------------------------------------------------------------
  d.nblk_jtj = (V + 255) / 256;
  d.jtj_group = prm->jtj_group;
  if (d.jtj_group == 0) {
    // by mesh size (fewer, fuller blocks for large meshes) and by the expected rows per 256 vertices:
    // about one vertex per covered pixel gets a correspondence and about half of those face the camera,
    // so rows ~ half the distinct pixels the template covers at its bind pose; sparse rows make a
    // block's partial cost more than its rows
    const int by_size = d.nblk_jtj <= 304 ? 1 : d.nblk_jtj <= 608 ? 2 : 4;
    std::vector<unsigned char> hit((size_t)W * H, 0);
    double covered = 0.0;
    for (int i = 0; i < V; ++i) {
      const double x = mesh->verts[3 * i], y = mesh->verts[3 * i + 1], z = mesh->verts[3 * i + 2];
      if (!(z > prm->z_near_m)) continue;
      const double u = std::floor(cam->fx * x / z + cam->cx + 0.5), v = std::floor(cam->fy * y / z + cam->cy + 0.5);
      if (u < 0 || v < 0 || u >= W || v >= H) continue;
      unsigned char& h = hit[(size_t)v * W + (size_t)u];
      if (!h) {
        h = 1;
        covered += 1.0;
      }
    }
    const double rows = 256.0 * 0.5 * covered / (double)V;  // ~3/4 of the rows measured on the test scenes
    const int by_rows = rows < 18.0 ? 4 : rows < 30.0 ? 2 : 1;
    d.jtj_group = std::max(by_size, by_rows);
  }
  d.nblk_rows = (d.nblk_jtj + d.jtj_group - 1) / d.jtj_group;
  d.nblk_v = (V + 255) / 256;
  carve_all(s);
  {  // the arena's size on the device: the carved bytes rounded up to the allocation granularity
    const size_t g = vmm_granularity();
    if (!g) return fail(TRK_ERR_CUDA, "the driver's virtual memory management is not available");
    s->device_bytes = (std::max<size_t>(s->carved, 1) + g - 1) / g * g;
  }
  CK(cudaMallocHost(&s->h_pinned, sizeof(double) * (L + prm->pose_iters + prm->shape_iters + 4)));
  CK(cudaMallocHost(&s->h_phi, sizeof(float4) * std::max(V, 1)));
  // the state of trk_set_pose(Theta = 0, Phi = 0)
  s->ev_theta.assign(L, 0.0);
  s->ev_lam = prm->lambda_k0;
  s->ev_phi.assign(V, make_float4(0.f, 0.f, 0.f, 0.f));
  s->frames_done = 0;
  if (resident) TRY(materialize(s));
  *out = s;
  s = nullptr;  // disarm the guard
  return TRK_OK;
}

}  // namespace

extern "C" {

trk_status trk_create(const trk_mesh* mesh, const trk_skeleton* sk, const trk_intrinsics* cam, const trk_params* prm,
                      trk_session** out) {
  return create_session(mesh, sk, cam, prm, true, out);
}

trk_status trk_create_evicted(const trk_mesh* mesh, const trk_skeleton* sk, const trk_intrinsics* cam,
                              const trk_params* prm, trk_session** out) {
  return create_session(mesh, sk, cam, prm, false, out);
}

trk_status trk_session_evict(trk_session* s) {
  NvtxRange nv("trk_session_evict");
  if (!s) return fail(TRK_ERR_INVALID_ARG, "NULL session");
  return evict(s);
}

trk_status trk_session_restore(trk_session* s) {
  NvtxRange nv("trk_session_restore");
  if (!s) return fail(TRK_ERR_INVALID_ARG, "NULL session");
  return materialize(s);
}

int32_t trk_session_is_resident(const trk_session* s) { return s && s->resident ? 1 : 0; }

trk_status trk_fk_joint_positions(const trk_skeleton* sk, const double* theta, double* out) {
  if (!sk || !theta || !out || sk->n_links < 1 || sk->n_links > TRK_MAX_LINKS || !sk->parent || !sk->type ||
      !sk->axis || !sk->offset_dq)
    return fail(TRK_ERR_INVALID_ARG, "trk_fk_joint_positions: bad arguments");
  const int L = sk->n_links;
  std::vector<HDQ> H(L);
  for (int j = 0; j < L; ++j) {
    const int p = sk->parent[j];
    if (p >= j) return fail(TRK_ERR_INVALID_ARG, "trk_fk_joint_positions: parent %d of link %d", p, j);
    const float* a = sk->axis + 3 * j;
    const double an = std::sqrt((double)a[0] * a[0] + (double)a[1] * a[1] + (double)a[2] * a[2]);
    const double ax = a[0] / an, ay = a[1] / an, az = a[2] / an;
    HDQ J{{1, 0, 0, 0}, {0, 0, 0, 0}};
    if (sk->type[j] == 0) {  // hinge: rotation by theta about the axis
      const double c = std::cos(0.5 * theta[j]), sn = std::sin(0.5 * theta[j]);
      J.r = {c, sn * ax, sn * ay, sn * az};
    } else {  // prismatic: translation by theta along the axis
      J.d = {0, 0.5 * theta[j] * ax, 0.5 * theta[j] * ay, 0.5 * theta[j] * az};
    }
    const float* o = sk->offset_dq + 8 * j;
    const HDQ off{{o[0], o[1], o[2], o[3]}, {o[4], o[5], o[6], o[7]}};
    const HDQ base = p < 0 ? HDQ{{1, 0, 0, 0}, {0, 0, 0, 0}} : H[p];
    H[j] = hdmul(hdmul(base, off), J);
    // translation of a unit dual quaternion: 2 vec(d r*)
    const HQ rc{H[j].r.w, -H[j].r.x, -H[j].r.y, -H[j].r.z};
    const HQ t = hmul(H[j].d, rc);
    const double n2 = H[j].r.w * H[j].r.w + H[j].r.x * H[j].r.x + H[j].r.y * H[j].r.y + H[j].r.z * H[j].r.z;
    out[3 * j] = 2 * t.x / n2;
    out[3 * j + 1] = 2 * t.y / n2;
    out[3 * j + 2] = 2 * t.z / n2;
  }
  return TRK_OK;
}

trk_status trk_set_pose(trk_session* s, const double* theta, const float* offsets) {
  if (!s || !theta) return fail(TRK_ERR_INVALID_ARG, "NULL argument");
  Dev& d = s->d;
  for (int j = 0; j < d.L; ++j)
    if (!std::isfinite(theta[j])) return fail(TRK_ERR_NUMERIC, "theta[%d] not finite", j);
  s->frames_done = 0;  // a new sequence starts (shape-match fits the shape on its first frame)
  std::vector<float4> phi(d.V, make_float4(0.f, 0.f, 0.f, 0.f));
  if (offsets)
    for (int i = 0; i < d.V; ++i) {
      if (!std::isfinite(offsets[3 * i]) || !std::isfinite(offsets[3 * i + 1]) || !std::isfinite(offsets[3 * i + 2]))
        return fail(TRK_ERR_NUMERIC, "offset %d not finite", i);
      phi[i] = make_float4(offsets[3 * i], offsets[3 * i + 1], offsets[3 * i + 2], 0.f);
    }
  const double lam = s->prm.lambda_k0;
  if (!s->resident) {  // the state waits on the host until the session is restored
    s->ev_theta.assign(theta, theta + d.L);
    s->ev_phi = phi;
    s->ev_lam = lam;
    return TRK_OK;
  }
  CK(cudaMemcpyAsync(d.theta, theta, sizeof(double) * d.L, cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemcpyAsync(d.phi[0], phi.data(), sizeof(float4) * d.V, cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemcpyAsync(d.lam, &lam, sizeof(double), cudaMemcpyHostToDevice, s->stream));
  launch_fk(d, s->stream);
  return sync_check(s);
}

namespace {
struct CheckpointHeader {
  char magic[8];
  int32_t version, n_links, n_verts, frames_done;
};
static_assert(sizeof(CheckpointHeader) == 24, "checkpoint header layout");
constexpr char kCheckpointMagic[8] = {'T', 'R', 'K', 'S', 'T', 'A', 'T', 'E'};
constexpr int32_t kCheckpointVersion = 1;

size_t checkpoint_bytes(const Dev& d) {
  return sizeof(CheckpointHeader) + sizeof(double) * ((size_t)d.L + 1) + sizeof(float4) * (size_t)d.V;
}
}  // namespace

trk_status trk_session_export(trk_session* s, void* blob, size_t* size_bytes) {
  if (!s || !size_bytes) return fail(TRK_ERR_INVALID_ARG, "NULL argument");
  const Dev& d = s->d;
  const size_t need = checkpoint_bytes(d);
  if (!blob) {
    *size_bytes = need;
    return TRK_OK;
  }
  if (*size_bytes < need) return fail(TRK_ERR_INVALID_ARG, "checkpoint buffer of %zu bytes, %zu needed", *size_bytes, need);
  CheckpointHeader h{};
  std::memcpy(h.magic, kCheckpointMagic, sizeof(h.magic));
  h.version = kCheckpointVersion;
  h.n_links = d.L;
  h.n_verts = d.V;
  h.frames_done = s->frames_done;
  unsigned char* p = static_cast<unsigned char*>(blob);
  std::memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  if (!s->resident) {
    std::memcpy(p, s->ev_theta.data(), sizeof(double) * d.L);
    std::memcpy(p + sizeof(double) * d.L, &s->ev_lam, sizeof(double));
    std::memcpy(p + sizeof(double) * (d.L + 1), s->ev_phi.data(), sizeof(float4) * d.V);
    *size_bytes = need;
    return TRK_OK;
  }
  // on the stream of the last frame, so that the copies follow it
  cudaStream_t st = s->last_stream ? s->last_stream : s->stream;
  CK(cudaMemcpyAsync(p, d.theta, sizeof(double) * d.L, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(p + sizeof(double) * d.L, d.lam, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(p + sizeof(double) * (d.L + 1), d.phi[0], sizeof(float4) * d.V, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  s->last_stream = nullptr;
  *size_bytes = need;
  return TRK_OK;
}

trk_status trk_session_import(trk_session* s, const void* blob, size_t size_bytes) {
  if (!s || !blob) return fail(TRK_ERR_INVALID_ARG, "NULL argument");
  Dev& d = s->d;
  CheckpointHeader h;
  if (size_bytes < sizeof(h)) return fail(TRK_ERR_INVALID_ARG, "checkpoint of %zu bytes is too short", size_bytes);
  std::memcpy(&h, blob, sizeof(h));
  if (std::memcmp(h.magic, kCheckpointMagic, sizeof(h.magic)) != 0 || h.version != kCheckpointVersion)
    return fail(TRK_ERR_INVALID_ARG, "not a session checkpoint of format version %d", kCheckpointVersion);
  if (h.n_links != d.L || h.n_verts != d.V)
    return fail(TRK_ERR_INVALID_ARG, "checkpoint of a model with %d links and %d vertices; the session has %d and %d",
                h.n_links, h.n_verts, d.L, d.V);
  const size_t need = checkpoint_bytes(d);
  if (size_bytes != need) return fail(TRK_ERR_INVALID_ARG, "checkpoint of %zu bytes, %zu expected", size_bytes, need);
  if (h.frames_done < 0) return fail(TRK_ERR_INVALID_ARG, "checkpoint frame count %d", h.frames_done);
  const unsigned char* p = static_cast<const unsigned char*>(blob) + sizeof(h);
  std::vector<double> th(d.L + 1);  // Theta, then lambda
  std::memcpy(th.data(), p, sizeof(double) * (d.L + 1));
  std::vector<float4> phi(d.V);
  std::memcpy(phi.data(), p + sizeof(double) * (d.L + 1), sizeof(float4) * d.V);
  for (int j = 0; j < d.L; ++j)
    if (!std::isfinite(th[j])) return fail(TRK_ERR_NUMERIC, "checkpoint theta[%d] not finite", j);
  if (!std::isfinite(th[d.L]) || !(th[d.L] > 0.0)) return fail(TRK_ERR_NUMERIC, "checkpoint lambda %g", th[d.L]);
  for (int i = 0; i < d.V; ++i)
    if (!std::isfinite(phi[i].x) || !std::isfinite(phi[i].y) || !std::isfinite(phi[i].z))
      return fail(TRK_ERR_NUMERIC, "checkpoint offset %d not finite", i);
  if (!s->resident) {
    s->ev_theta.assign(th.begin(), th.begin() + d.L);
    s->ev_lam = th[d.L];
    s->ev_phi = phi;
    s->frames_done = h.frames_done;
    return TRK_OK;
  }
  if (s->last_stream) CK(cudaStreamSynchronize(s->last_stream));  // the last frame still reads the state
  s->last_stream = nullptr;
  CK(cudaMemcpyAsync(d.theta, th.data(), sizeof(double) * d.L, cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemcpyAsync(d.lam, th.data() + d.L, sizeof(double), cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemcpyAsync(d.phi[0], phi.data(), sizeof(float4) * d.V, cudaMemcpyHostToDevice, s->stream));
  launch_fk(d, s->stream);  // H_{j,Delta} and the twists of Theta, as after the frame that wrote them
  s->frames_done = h.frames_done;
  return sync_check(s);
}

trk_status trk_track_frame(trk_session* s, const float* depth_m, trk_result* out) {
  NvtxRange nv("trk_track_frame");
  if (!s || !depth_m) return fail(TRK_ERR_INVALID_ARG, "NULL argument");
  NEED_RESIDENT(s);
  cudaGraphExec_t ge;
  TRY(frame_graph(s, &ge));
  const Dev& d = s->d;
  CK(cudaMemcpyAsync(const_cast<float*>(d.depth), depth_m, sizeof(float) * d.cam.W * d.cam.H, cudaMemcpyHostToDevice,
                     s->stream));
  launch_tiles(d, d.depth, s->stream);  // the frame's occupied tiles (the graph's association reads them)
  CK(cudaGraphLaunch(ge, s->stream));
  ++s->frames_done;
  s->last_stream = s->stream;
  TRY(fetch_result(s, s->stream, out));
  return sync_check(s);
}

trk_status trk_track_frame_device(trk_session* s, const float* d_depth_m, void* cuda_stream) {
  NvtxRange nv("trk_track_frame_device");
  if (!s || !d_depth_m) return fail(TRK_ERR_INVALID_ARG, "NULL argument");
  NEED_RESIDENT(s);
  cudaGraphExec_t ge;
  TRY(frame_graph(s, &ge));
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : s->stream;
  launch_tiles(s->d, d_depth_m, st);  // copies the caller's depth and lists its occupied tiles: no memcpy
  CK(cudaGraphLaunch(ge, st));
  ++s->frames_done;
  CK(cudaGetLastError());
  s->last_stream = st;
  return TRK_OK;
}

trk_status trk_read_result(trk_session* s, trk_result* out) {
  if (!s) return fail(TRK_ERR_INVALID_ARG, "NULL argument");
  NEED_RESIDENT(s);
  cudaStream_t st = s->last_stream ? s->last_stream : s->stream;
  TRY(fetch_result(s, st, out));
  CK(cudaGetLastError());
  s->last_stream = nullptr;  // the frame is done: nothing left to wait for on that stream
  return TRK_OK;
}

trk_status trk_render_depth(trk_session* s, const double* theta, const float* offsets, float* depth_m) {
  if (!s || !theta || !depth_m) return fail(TRK_ERR_INVALID_ARG, "NULL argument");
  NEED_RESIDENT(s);
  Dev r = s->d;  // scratch view: FK tables and offsets in candidate / sweep buffers, state untouched
  r.theta = s->d.theta_c;
  r.Hd = s->d.Hd_c;
  r.xi = s->d.xi_c;
  r.phi[0] = s->d.phi0;
  std::vector<float4> phi(r.V, make_float4(0.f, 0.f, 0.f, 0.f));
  if (offsets)
    for (int i = 0; i < r.V; ++i) phi[i] = make_float4(offsets[3 * i], offsets[3 * i + 1], offsets[3 * i + 2], 0.f);
  CK(cudaMemcpyAsync(r.theta, theta, sizeof(double) * r.L, cudaMemcpyHostToDevice, s->stream));
  CK(cudaMemcpyAsync(r.phi[0], phi.data(), sizeof(float4) * r.V, cudaMemcpyHostToDevice, s->stream));
  launch_fk(r, s->stream);
  launch_skin(r, 0, s->stream);
  launch_raster(r, s->stream);
  launch_depth_from_zbuf(r, s->d_render, s->stream);
  CK(cudaMemcpyAsync(depth_m, s->d_render, sizeof(float) * r.cam.W * r.cam.H, cudaMemcpyDeviceToHost, s->stream));
  return sync_check(s);
}

trk_status trk_set_depth(trk_session* s, const float* depth_m) {
  if (!s || !depth_m) return fail(TRK_ERR_INVALID_ARG, "NULL argument");
  NEED_RESIDENT(s);
  CK(cudaMemcpyAsync(const_cast<float*>(s->d.depth), depth_m, sizeof(float) * s->d.cam.W * s->d.cam.H,
                     cudaMemcpyHostToDevice, s->stream));
  launch_tiles(s->d, s->d.depth, s->stream);
  return sync_check(s);
}

trk_status trk_step_skin(trk_session* s) {
  if (!s) return fail(TRK_ERR_INVALID_ARG, "NULL session");
  NEED_RESIDENT(s);
  launch_fk(s->d, s->stream);
  launch_skin(s->d, 0, s->stream);
  return sync_check(s);
}
trk_status trk_step_raster(trk_session* s) {
  if (!s) return fail(TRK_ERR_INVALID_ARG, "NULL session");
  NEED_RESIDENT(s);
  launch_raster(s->d, s->stream);
  return sync_check(s);
}
trk_status trk_step_visibility(trk_session* s) {
  if (!s) return fail(TRK_ERR_INVALID_ARG, "NULL session");
  NEED_RESIDENT(s);
  // empty buckets first, so that calling this step twice cannot insert a vertex twice
  CK(cudaMemsetAsync(s->d.head, 0xFF, sizeof(int) * s->d.cam.W * s->d.cam.H, s->stream));
  launch_visibility(s->d, s->stream);
  return sync_check(s);
}
trk_status trk_step_associate(trk_session* s) {
  if (!s) return fail(TRK_ERR_INVALID_ARG, "NULL session");
  NEED_RESIDENT(s);
  CK(cudaMemsetAsync(s->d.qctl, 0, sizeof(unsigned) * 2, s->stream));
  launch_associate(s->d, s->stream);
  return sync_check(s);
}
trk_status trk_step_normal_equations(trk_session* s) {
  if (!s) return fail(TRK_ERR_INVALID_ARG, "NULL session");
  NEED_RESIDENT(s);
  launch_normal_equations(s->d, 0, 0, s->stream);
  return sync_check(s);
}
trk_status trk_step_lm(trk_session* s) {
  if (!s) return fail(TRK_ERR_INVALID_ARG, "NULL session");
  NEED_RESIDENT(s);
  launch_lm(s->d, 0, s->stream);
  return sync_check(s);
}
trk_status trk_step_shape(trk_session* s) {
  if (!s) return fail(TRK_ERR_INVALID_ARG, "NULL session");
  NEED_RESIDENT(s);
  const int cur = launch_shape(s->d, 0, s->prm.pose_iters, s->stream);
  if (cur != 0)
    CK(cudaMemcpyAsync(s->d.phi[0], s->d.phi[cur], sizeof(float4) * s->d.V, cudaMemcpyDeviceToDevice, s->stream));
  return sync_check(s);
}

trk_status trk_read(trk_session* s, trk_field field, void* dst, size_t bytes) {
  if (!s || !dst) return fail(TRK_ERR_INVALID_ARG, "NULL argument");
  NEED_RESIDENT(s);
  const Dev& d = s->d;
  const size_t V = d.V, npx = (size_t)d.cam.W * d.cam.H, L = d.L, NP = d.NP;
  const void* src = nullptr;
  size_t need = 0;
  switch (field) {
    case TRK_FIELD_VERTS: src = d.v; need = V * 16; break;
    case TRK_FIELD_NORMALS: src = d.n; need = V * 16; break;
    case TRK_FIELD_ZBUF: src = d.zbuf; need = npx * 8; break;
    case TRK_FIELD_VISPIX: src = d.vispix; need = V * 4; break;
    case TRK_FIELD_CORR: src = d.corr; need = npx * 4; break;
    case TRK_FIELD_ACC: src = d.acc; need = V * 32; break;
    case TRK_FIELD_NORMAL_EQ: src = d.A; need = NP * NP * 8; break;
    case TRK_FIELD_THETA: src = d.theta; need = L * 8; break;
    case TRK_FIELD_PHI: src = d.phi[0]; need = V * 16; break;
    case TRK_FIELD_LAMBDA: src = d.lam; need = 8; break;
    case TRK_FIELD_ENERGY: src = d.energy; need = (size_t)(s->prm.pose_iters + s->prm.shape_iters) * 8; break;
    case TRK_FIELD_LM_TRIALS: src = d.lm_trials; need = 64; break;
    case TRK_FIELD_SHAPE_RG: src = d.rg; need = V * 16; break;
    case TRK_FIELD_NEIGHBOURS: src = d.nbr; need = V * 16; break;
    case TRK_FIELD_PRIOR: src = d.prior2; need = L * 8; break;
    case TRK_FIELD_LM_SOLVER: src = d.lm_ok + kCandidates; need = kCandidates * 4; break;
    default: return fail(TRK_ERR_INVALID_ARG, "unknown field %d", (int)field);
  }
  if (bytes != need) return fail(TRK_ERR_INVALID_ARG, "field %d needs %zu bytes, got %zu", (int)field, need, bytes);
  if (need) CK(cudaMemcpyAsync(dst, src, need, cudaMemcpyDeviceToHost, s->stream));
  TRY(sync_check(s));
  if (field == TRK_FIELD_VERTS) {  // session-local frame -> camera frame
    float4* v = static_cast<float4*>(dst);
    for (size_t i = 0; i < V; ++i) {
      v[i].x += d.cam.ox;
      v[i].y += d.cam.oy;
      v[i].z += d.cam.oz;
    }
  }
  return TRK_OK;
}

trk_status trk_get_info(trk_session* s, trk_info* out) {
  if (!s || !out) return fail(TRK_ERR_INVALID_ARG, "NULL argument");
  const Dev& d = s->d;
  out->n_links = d.L;
  out->n_verts = d.V;
  out->n_tris = d.F;
  out->width = d.cam.W;
  out->height = d.cam.H;
  const int per_assoc = (d.F > 0 ? 5 : 4);  // skin, raster, visibility, associate (2 kernels)
  const int shape_k = s->prm.shape_solver == 1 ? 3 * s->prm.shape_sweeps + 1 : s->prm.shape_sweeps;
  out->kernels_per_frame = 1 + s->prm.pose_iters * (per_assoc + 5) + s->prm.shape_iters * (per_assoc + shape_k);
  out->device_bytes = s->device_bytes;
  out->jtj_group = s->d.jtj_group;
  return TRK_OK;
}

trk_status trk_profile_iteration(trk_session* s, int32_t reps, size_t flush_bytes, float* ms) {
  if (!s || !ms || reps <= 0) return fail(TRK_ERR_INVALID_ARG, "bad argument");
  NEED_RESIDENT(s);
  const Dev& d = s->d;
  cudaStream_t st = s->stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  void* flush = nullptr;
  if (flush_bytes) CK(cudaMalloc(&flush, flush_bytes));
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
  cudaError_t err = cudaSuccess;
  for (int r = 0; r < reps && err == cudaSuccess; ++r) {
    err = timed(TRK_STAGE_SKIN, [&] { launch_skin(d, 0, st); });
    if (!err) err = timed(TRK_STAGE_RASTER, [&] { launch_raster(d, st); });
    if (!err) err = timed(TRK_STAGE_VISIBILITY, [&] { launch_visibility(d, st); });
    if (!err) err = timed(TRK_STAGE_ASSOCIATE, [&] { launch_associate(d, st); });
    if (!err) err = timed(TRK_STAGE_RESID_JTJ, [&] { launch_resid_jtj(d, 0, st); });
    if (!err) err = timed(TRK_STAGE_REDUCE, [&] { launch_reduce_jtj(d, -1, st); });
    if (!err) err = timed(TRK_STAGE_LM_SOLVE, [&] { launch_lm_solve(d, st); });
    if (!err) err = timed(TRK_STAGE_LM_EVAL, [&] { launch_lm_eval(d, 0, st); });
  }
  for (int r = 0; r < reps && err == cudaSuccess; ++r) {
    launch_skin(d, 0, st);
    launch_raster(d, st);
    launch_visibility(d, st);
    launch_associate(d, st);
    int cur = 0;
    err = timed(TRK_STAGE_SHAPE, [&] { cur = launch_shape(d, 0, -1, st); });
    if (!err && cur != 0) err = cudaMemcpyAsync(d.phi[0], d.phi[cur], sizeof(float4) * d.V, cudaMemcpyDeviceToDevice, st);
  }
  cudaStreamSynchronize(st);
  if (flush) cudaFree(flush);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(err);
  for (int k = 0; k < TRK_STAGE_COUNT; ++k) ms[k] = (float)(acc[k] / reps);
  return TRK_OK;
}

}  // extern "C"
