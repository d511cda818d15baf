// trk_internal.cuh -- device data layout and dual-quaternion arithmetic shared by the tracker's kernels.
//
// Layout in device memory (one session):
//   links      : LinkTable (parent, type, axis, offset DQ, conj(bind DQ)) -- a few KB, read into shared memory
//   per vertex : v0[V] float4, phi[2][V] float4 (Jacobi double buffer), bones[V] (uchar4 idx + float4 w),
//                v[V] float4, n[V] float4 (w = valid), rec[V] float4 (x,y,z, next-in-bucket bits),
//                acc[V] Acc4 (sum of p_k - v_i in 2^-30 m, count), vispix[V] int, nbr[V] int4, rg[V] float4
//   per face   : tris[F] int4 (a,b,c,pad), fn[F] float4 face normals
//   per pixel  : depth[W*H] float, zbuf[W*H] u64, head[W*H] int, corr[W*H] int
//   solver     : partials[nblk][NP*NP] float, A[NP*NP] double, per-candidate theta / DQ tables
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/trk.h"

namespace trk {

constexpr int kMaxLinks = 79;       // NP = P + 1 <= 80
constexpr int kMaxNP = 80;
constexpr int kMaxJtjGroup = 4;    // vertex blocks of 256 per [J r] block at most (trk_params.jtj_group)
constexpr int kUnitsPerTile = 8;   // association units (16 x 2 pixels) per 16 x 16 tile
constexpr int kAssocBlocksPerSM = 4;  // resident association blocks per SM (registers sized for it)
constexpr int kCandidates = 6;      // damping values tried per LM iteration: lambda * 10^c, c = 0..5
constexpr float kFix = 1073741824.0f;  // 2^30: fixed-point scale of the per-vertex sums

struct DQ {
  float4 r, d;  // (w, x, y, z) real and dual parts
};

// Per-vertex association sums: sum of (p_k - v_i) in units of 2^-30 m, and the pixel count.
struct __align__(32) Acc4 {
  long long x, y, z, w;
};

// All positions on the device live in a session-local frame: the camera frame shifted by the template's
// bind-pose centroid c (so coordinates stay within ~1 m and FP32 keeps ~1e-7 m of absolute precision).
// FK starts from pre = T(-c); the bind pose is stored in the same frame.
struct LinkTable {
  int L;
  int max_depth;  // largest link depth (root links: 0)
  int depth[kMaxLinks];
  int parent[kMaxLinks];
  int type[kMaxLinks];
  float axis[kMaxLinks][3];
  // The links split into chains: a link continues its parent's chain when it is the parent's only
  // child, else it starts a chain.  chain[] lists the links chain by chain, each from its head down;
  // chain c is chain[chain_start[c] .. chain_start[c + 1]).  Chains are grouped in rounds: a chain's
  // round is one more than the round of the chain holding its head's parent (root chains: round 0), and
  // round r holds chains round_start[r] .. round_start[r + 1] - 1.
  int n_chains, n_rounds;
  int chain[kMaxLinks];
  int chain_start[kMaxLinks + 1];
  int round_start[kMaxLinks + 1];
  DQ pre;               // T(-c)
  DQ off[kMaxLinks];
  DQ bindc[kMaxLinks];  // conjugate of the bind-pose DQ T(-c) H^0_{0,j}
};
static_assert(sizeof(LinkTable) % 16 == 0, "LinkTable is copied in 16-byte units");

// Per-session constants passed by value to the kernels.
struct Cam {
  int W, H;
  float fx, fy, cx, cy;
  float z_near, eps_vis, tau, kappa;  // kappa: ring-bound factor of the association search
  int R;                               // window half-size
  float ox, oy, oz;                    // origin c of the session-local frame (camera coordinates)
  double inv_fx, inv_fy;
};

// ---------------------------------------------------------------------------------------------
// quaternion / dual quaternion arithmetic (FP32)
// ---------------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ float4 qmul(float4 a, float4 b) {
  return make_float4(a.x * b.x - a.y * b.y - a.z * b.z - a.w * b.w,
                     a.x * b.y + a.y * b.x + a.z * b.w - a.w * b.z,
                     a.x * b.z - a.y * b.w + a.z * b.x + a.w * b.y,
                     a.x * b.w + a.y * b.z - a.z * b.y + a.w * b.x);
}
__host__ __device__ __forceinline__ float4 qconj(float4 a) { return make_float4(a.x, -a.y, -a.z, -a.w); }
__host__ __device__ __forceinline__ float4 qadd(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__host__ __device__ __forceinline__ float4 qscale(float4 a, float s) {
  return make_float4(a.x * s, a.y * s, a.z * s, a.w * s);
}
__host__ __device__ __forceinline__ float qdot(float4 a, float4 b) {
  return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}
__host__ __device__ __forceinline__ DQ dqmul(const DQ& a, const DQ& b) {
  DQ h;
  h.r = qmul(a.r, b.r);
  h.d = qadd(qmul(a.r, b.d), qmul(a.d, b.r));
  return h;
}
__host__ __device__ __forceinline__ DQ dqconj(const DQ& a) {
  DQ h;
  h.r = qconj(a.r);
  h.d = qconj(a.d);
  return h;
}

// joint transform of link j at value th (hinge: rotation about z; prismatic: translation along z)
__device__ __forceinline__ DQ joint_dq(int type, const float* z, float th) {
  DQ h;
  if (type == 0) {
    float s, c;
    sincosf(0.5f * th, &s, &c);
    h.r = make_float4(c, z[0] * s, z[1] * s, z[2] * s);
    h.d = make_float4(0.f, 0.f, 0.f, 0.f);
  } else {
    h.r = make_float4(1.f, 0.f, 0.f, 0.f);
    h.d = make_float4(0.f, 0.5f * th * z[0], 0.5f * th * z[1], 0.5f * th * z[2]);
  }
  return h;
}

// Asynchronous global -> shared copies (cp.async); cp_async_wait_all() waits for all of this thread's.
__device__ __forceinline__ void cp_async8(void* s, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((uint32_t)__cvta_generic_to_shared(s)),
               "l"(__cvta_generic_to_global(g))
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* s, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((uint32_t)__cvta_generic_to_shared(s)),
               "l"(__cvta_generic_to_global(g))
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Forward kinematics of all links (Sec. 3.1): H_{0,j} = H_{0,parent(j)} off_j J_j(theta_j) (H_{0,-1} = the
// root transform pre), formed as (H_{0,parent} off_j) J_j.  Writes H_{j,Delta} = H_{0,j} conj(H^0_{0,j})
// and the twist Xi_j = H_{0,j} G_j conj(H_{0,j}) with G_j = (0, z/2 | 0) for a hinge and (0 | 0, z/2) for
// a prismatic joint (the joint's generator H_j^{-1} dH_j/dtheta_j): dH_{k,Delta}/dtheta_j = Xi_j H_{k,Delta}
// for every k below j.
//
// One thread walks each chain of single-child links (a 3-DoF joint is three such links), the chains of a
// round in parallel, one barrier per round: the products are those of a link-by-link walk from the root,
// with ~3x fewer barriers.  H0 (shared, [L]) is scratch; all threads of the block must call it.
template <typename ThetaT>
__device__ __forceinline__ void fk_all(const LinkTable& lt, const ThetaT* theta, DQ* H0, DQ* Hd_out, float* xi_out,
                                       int xi_stride) {
  const int L = lt.L;
  for (int j = threadIdx.x; j < L; j += blockDim.x) H0[j] = joint_dq(lt.type[j], lt.axis[j], (float)theta[j]);
  __syncthreads();
  for (int r = 0; r < lt.n_rounds; ++r) {
    for (int c = lt.round_start[r] + threadIdx.x; c < lt.round_start[r + 1]; c += blockDim.x) {
      const int head = lt.chain[lt.chain_start[c]];
      DQ H = lt.parent[head] < 0 ? lt.pre : H0[lt.parent[head]];
      for (int t = lt.chain_start[c]; t < lt.chain_start[c + 1]; ++t) {
        const int j = lt.chain[t];
        H = dqmul(dqmul(H, lt.off[j]), H0[j]);
        H0[j] = H;
      }
    }
    __syncthreads();
  }
  for (int j = threadIdx.x; j < L; j += blockDim.x) {
    const DQ H = H0[j];
    Hd_out[j] = dqmul(H, lt.bindc[j]);
    DQ G;
    const float* z = lt.axis[j];
    if (lt.type[j] == 0) {
      G.r = make_float4(0.f, 0.5f * z[0], 0.5f * z[1], 0.5f * z[2]);
      G.d = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
      G.r = make_float4(0.f, 0.f, 0.f, 0.f);
      G.d = make_float4(0.f, 0.5f * z[0], 0.5f * z[1], 0.5f * z[2]);
    }
    const DQ X = dqmul(dqmul(H, G), dqconj(H));
    float* xo = xi_out + (size_t)j * xi_stride;
    xo[0] = X.r.y; xo[1] = X.r.z; xo[2] = X.r.w;
    xo[3] = X.d.y; xo[4] = X.d.z; xo[5] = X.d.w;
    if (xi_stride > 6) { xo[6] = 0.f; xo[7] = 0.f; }
  }
}

// Blend of the <= 4 bone offsets of a vertex with the antipodal sign alignment to the heaviest bone
// (largest weight, ties to the smaller link index).
__device__ __forceinline__ DQ blend_bones(const DQ* Hd, uchar4 bi, float4 bw, float sg[4]) {
  const int idx[4] = {bi.x, bi.y, bi.z, bi.w};
  const float w[4] = {bw.x, bw.y, bw.z, bw.w};
  int js = -1;
  float wst = -1.f;
#pragma unroll
  for (int s = 0; s < 4; ++s)
    if (w[s] > 0.f && (w[s] > wst || (w[s] == wst && idx[s] < js))) { wst = w[s]; js = idx[s]; }
  const float4 ref = Hd[js < 0 ? 0 : js].r;
  DQ acc;
  acc.r = make_float4(0.f, 0.f, 0.f, 0.f);
  acc.d = acc.r;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    sg[s] = 0.f;
    if (!(w[s] > 0.f)) continue;
    const DQ h = Hd[idx[s]];
    const float g = qdot(h.r, ref) >= 0.f ? 1.f : -1.f;
    sg[s] = g;
    acc.r = qadd(acc.r, qscale(h.r, w[s] * g));
    acc.d = qadd(acc.d, qscale(h.d, w[s] * g));
  }
  return acc;
}

// Homogeneous point map of a (non-unit) blended DQ: (vec(a x a*) + 2 vec(b a*)) / |a|^2.
__device__ __forceinline__ float3 dq_point(const DQ& H, float3 x) {
  const float4 a = H.r, b = H.d;
  const float N = qdot(a, a);
  const float4 X = make_float4(0.f, x.x, x.y, x.z);
  const float4 t1 = qmul(qmul(a, X), qconj(a));
  const float4 t2 = qmul(b, qconj(a));
  const float inv = 1.f / N;
  return make_float3((t1.y + 2.f * t2.y) * inv, (t1.z + 2.f * t2.z) * inv, (t1.w + 2.f * t2.w) * inv);
}

// ---------------------------------------------------------------------------------------------
// launchers (defined in the kernel translation units)
// ---------------------------------------------------------------------------------------------
struct Dev;  // device pointers of one session, defined below
void launch_fk(const Dev& d, cudaStream_t st);
void launch_skin(const Dev& d, int phi_buf, cudaStream_t st);
void launch_raster(const Dev& d, cudaStream_t st);
void launch_visibility(const Dev& d, cudaStream_t st);
void launch_associate(const Dev& d, cudaStream_t st);  // two kernels: thread-owned rings, then the queue
// Device memory straight from the driver's virtual memory management, for what the library holds while
// running (session arenas, the frame server's step buffers): physical memory in units of the allocation
// granularity (2 MiB here) mapped into a reserved address range.  A block holds exactly its size rounded
// up to the granularity, and freeing it returns the memory to the device at once -- no pool keeps it.
// vmm_alloc: on the current device; *size receives the rounded size.  vmm_free: the memory must be idle.
struct VmmBlock {
  void* ptr = nullptr;
  size_t size = 0;
  unsigned long long handle = 0;
};
size_t vmm_granularity();  // of the current device (0 if the driver's API is unavailable)
cudaError_t vmm_alloc(size_t bytes, VmmBlock* out);
void vmm_free(VmmBlock* b);
size_t vmm_bytes_held();   // bytes the library holds through vmm_alloc now, over all devices
// Copies the frame's depth from src into d.depth (src == d.depth: in place), marks every pixel "no
// correspondence" and lists the association units (16 x 2 pixels) that hold a valid pixel (the
// single-session association takes its units from that list).
void launch_tiles(const Dev& d, const float* src, cudaStream_t st);
// residual + Jacobian + [J r]^T [J r]; writes E_pose to energy[slot] (slot < 0: not recorded)
void launch_normal_equations(const Dev& d, int phi_buf, int slot, cudaStream_t st);
void launch_lm(const Dev& d, int phi_buf, cudaStream_t st);
// the same kernels one at a time (used by the per-kernel timing)
void launch_resid_jtj(const Dev& d, int phi_buf, cudaStream_t st);
void launch_reduce_jtj(const Dev& d, int slot, cudaStream_t st);
void launch_lm_solve(const Dev& d, cudaStream_t st);
void launch_lm_eval(const Dev& d, int phi_buf, cudaStream_t st);
// shape step from buffer phi_src; writes E_shape to energy[slot]; returns the buffer holding Phi after it
int launch_shape(const Dev& d, int phi_src, int slot, cudaStream_t st);
void launch_depth_from_zbuf(const Dev& d, float* out, cudaStream_t st);
void configure_kernels();
void ensure_configured();  // configure_kernels once per device (thread-safe)

// Records msg as this thread's last error (read by trk_last_error) and returns st.
int set_error_code(int st, const char* msg);
template <typename S>
inline S set_error(S st, const char* msg) { return static_cast<S>(set_error_code(static_cast<int>(st), msg)); }

}  // namespace trk

namespace trk {

// A warp's share of the association: up to 32 pixels of one 16 x 16 tile that hold a valid depth, in
// row-major order (lane l takes pixel (x0 + off[l] % 16, y0 + off[l] / 16) for l < n).
struct __align__(16) AssocUnit {
  int session, x0, y0, n;
  unsigned char off[32];
};

// Device pointers and constants of one session (passed by value to every kernel).
struct Dev {
  int V, F, L, NP;  // NP = L + 1 (the residual column of [J r])
  int pose_iters, shape_iters, shape_sweeps, knn;
  float lambda_phi, lambda_N, lambda_w;
  Cam cam;
  const LinkTable* links;
  // template and derived mesh data
  const float4* v0;
  const uchar4* bidx;
  const float4* bw;
  const int4* tris;
  const int* csr_off;
  const int* csr_face;
  const int4* nbr;
  const double* prior2;  // (lambda_s S_kk)^2
  // tracking state
  float4* phi[2];
  double* theta;
  double* lam;
  double* energy;
  DQ* Hd;
  float* xi;  // [L][8], 6 used
  // LM candidates
  double* theta_c;  // [kCandidates][L]
  DQ* Hd_c;         // [kCandidates][L]
  float* xi_c;      // [kCandidates][L][8]
  double* lm_trials;  // [8]
  int* lm_ok;         // [kCandidates] ok flags, then [kCandidates] solver diagnostics
  // per-iteration buffers
  float4* v;
  float4* n;
  float4* fn;
  float4* rec;
  float4* pixrec;  // [W*H] first vertex inserted into each pixel's bucket: x, y, z, index bits
  int* head;
  int4* queue;     // [W*H] pixels whose association search continues past the thread-owned rings
  unsigned int* qctl;  // [0] queued pixels, [1] next queue entry to take, [2] association units, [3] unused
  AssocUnit* units;  // [8 ceil(W/16) ceil(H/16)] association units of the frame (up to 32 valid pixels of a tile)
  unsigned long long* zbuf;
  int* corr;
  Acc4* acc;
  int* vispix;
  float4* rg;
  float4* phi0;
  const float* depth;
  // reductions
  float* partial;   // [nblk_rows][NP*NP]
  int jtj_group;    // 256-vertex blocks per [J r] block (1, 2 or 4)
  int nblk_rows;    // [J r] blocks: ceil(nblk_jtj / jtj_group)
  int* jtj_rows;    // [nblk_rows] rows of [J r] each block contributed (0: its partial is not written)
  float4* arec;     // [nblk_jtj * 256][4] per row of [J r]: what the candidate energies need of its vertex
  int nblk_jtj;
  double* A;        // [NP*NP]
  double* epart;    // [nblk_v][8]
  int nblk_v;
  unsigned int* counter;  // [4] last-block tickets
  int* stats;             // [0] associated pixels, [1] associated vertices, [3] tensor-core wait ran out
  int precision;          // TRK_PRECISION_*: arithmetic of [J r]^T [J r]
  int shape_solver;       // 0 Jacobi sweeps, 1 coupled PCG
  int association;        // 0 window search, 1 nearest corner of the rasterised triangle
  const int* adj_off;     // [V + 1] neighbourhood edges of each vertex in both directions (CSR) ...
  const int* adj;         // ... sorted by vertex index
  float4 *cg_x, *cg_r, *cg_z, *cg_p, *cg_ap;  // [V] PCG vectors
  double* cg;             // [4] rz, alpha, beta, stopped
};

}  // namespace trk

namespace trk {

// A named range on the host timeline of a profiler (NVTX; costs nothing when no profiler is attached):
// the C entry points and the stages a frame enqueues.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Warps that add one session's [J r] block partials: about four partials each (one round of loads), at
// most 32; a batched launch gives every block the largest count of its sessions (a block uses its own).
__host__ __device__ inline int reduce_warps(int nblk_rows) { return max(1, min(32, (nblk_rows + 3) / 4)); }

struct BatchGrid;
// Batched launches: one launch runs a stage for every session of a batch (block tables built by the batch).
void launch_skin_b(const BatchGrid& g, int nblk, int max_links, int phi_buf, unsigned* ctl, cudaStream_t st);
void launch_raster_b(const BatchGrid& g, int nblk, cudaStream_t st);
void launch_visibility_b(const BatchGrid& g, int nblk, cudaStream_t st);
void launch_associate_b(const Dev* devs, int n_sessions, const AssocUnit* units, unsigned* ctl, unsigned* prefix,
                        int assoc_blocks, int tail_blocks, cudaStream_t st);
void launch_gather_depth_b(const BatchGrid& g, int nblk, const float* const* srcs, AssocUnit* units, unsigned* ctl,
                           cudaStream_t st);
void launch_normal_equations_b(const BatchGrid* gj, const int* nj, const BatchGrid& gr, int nr, int max_links,
                               int precision, int phi_buf, int slot, cudaStream_t st, int reduce_threads);
void launch_lm_b(const BatchGrid& glm, int nlm, const BatchGrid& gv, int nv, int max_links, int phi_buf,
                 cudaStream_t st);
int launch_shape_b(const BatchGrid& gv, int nv, int max_links, int sweeps, int solver, int phi_src, int slot,
                   cudaStream_t st);

// Position of a block within its session's grid.  The single-session kernels take it from blockIdx and
// gridDim; the batched kernels (one launch over the blocks of many sessions) from a per-launch table.
struct BlockPos {
  int x, y, gx;
};
__device__ __forceinline__ BlockPos grid_pos() { return BlockPos{(int)blockIdx.x, (int)blockIdx.y, (int)gridDim.x}; }

// A batched launch: block b works for session map[b].x at position (map[b].y, map[b].z) of a grid of
// map[b].w blocks along x.
struct BatchGrid {
  const Dev* devs;
  const int4* map;
};

// Where a batched step writes one session's results (device-accessible, e.g. host-mapped pinned memory).
struct ResultDst {
  double* theta;   // [L]
  float4* phi;     // [V] (x, y, z, 0)
  double* energy;  // [pose_iters + shape_iters]
  int* stats;      // [4]
};
struct BatchStep;
// device bytes one session adds to a step's buffer (a buffer holds at most twice its step's sum, rounded
// up to the allocation granularity)
size_t batch_step_bytes_of(const trk_session* s);
BatchStep* batch_step_create();
void batch_step_destroy(BatchStep* bs, cudaStream_t st);
// One frame of the n sessions (resident, same schedule, precision and mode TRACK) as one launch per
// stage on st: session k reads its depth from srcs[k] and its results go to dst[k] (both device-
// accessible host pointers are fine).  The step's buffers may be reused once the stream passed it.
trk_status batch_step_launch(BatchStep* bs, trk_session* const* ss, int n, const float* const* srcs,
                             const ResultDst* dst, cudaStream_t st);

// Every stage kernel serves one session (g.map == nullptr: the descriptor is the kernel parameter and the
// block's position its blockIdx) and batches (descriptor and position from the tables, the descriptor
// staged in shared memory).  The device code is compiled without implicit multiply-add contraction, so
// the two inlined copies of a stage body round identically: a session computes bit for bit the same
// alone and in a batch.
__device__ __forceinline__ BlockPos batch_block(const BatchGrid& g, Dev& sd) {
  const int4 m = g.map[blockIdx.x];
  const int* src = reinterpret_cast<const int*>(g.devs + m.x);
  for (int t = threadIdx.x; t < (int)(sizeof(Dev) / 4); t += blockDim.x) reinterpret_cast<int*>(&sd)[t] = src[t];
  __syncthreads();
  return BlockPos{m.y, m.z, m.w};
}
constexpr BatchGrid kSingle{nullptr, nullptr};
// Resident blocks per SM that a batch's launches of the streaming stages (raster, visibility, shape) size
// their registers for: their grids span many sessions, where occupancy hides the gathers' latency.
constexpr int kBatchMinBlocks = 7;

}  // namespace trk
