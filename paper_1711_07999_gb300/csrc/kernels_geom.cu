// kernels_geom.cu -- forward kinematics, skinning, z-buffer, visibility / buckets and projective
// association (Secs. 3.1-3.3, 4.1).  All streams are per-vertex, per-triangle or per-pixel and
// HBM/L2-bound; vertex and pixel records are float4 so that each thread issues 16-byte loads.
#include "trk_internal.cuh"

namespace trk {

constexpr int kBlock = 256;

__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// ---------------------------------------------------------------------------------------------
// Sec. 3.1: FK of the current Theta -> H_{j,Delta} and the joint twists Xi_j (one thread per link)
// ---------------------------------------------------------------------------------------------
__global__ void k_fk(Dev d) {
  __shared__ LinkTable lt;
  __shared__ DQ H0[kMaxLinks];
  for (int t = threadIdx.x; t < (int)(sizeof(LinkTable) / 4); t += blockDim.x)
    reinterpret_cast<int*>(&lt)[t] = reinterpret_cast<const int*>(d.links)[t];
  __syncthreads();
  fk_all(lt, d.theta, H0, d.Hd, d.xi, 8);
}

void launch_fk(const Dev& d, cudaStream_t st) { k_fk<<<1, 128, 0, st>>>(d); }

// ---------------------------------------------------------------------------------------------
// Eqs. H_Sigma, deformation: v_i = H_iSigma (v0_i + phi_i).  Also clears the per-pixel and
// per-vertex accumulators of this iteration (z-buffer, bucket heads, association sums).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void skin_impl(const Dev& d, BlockPos bp, int phi_buf) {
  extern __shared__ DQ sHd[];
  for (int j = threadIdx.x; j < d.L; j += blockDim.x) sHd[j] = d.Hd[j];
  __syncthreads();
  const int tid = bp.x * blockDim.x + threadIdx.x;
  const int stride = bp.gx * blockDim.x;
  const int npx = d.cam.W * d.cam.H;
  for (int k = tid; k < npx; k += stride) {  // (corr: set once per frame with the depth, see k_tiles)
    d.zbuf[k] = ~0ull;
    d.head[k] = -1;
  }
  for (int k = tid; k < d.V; k += stride) d.acc[k] = Acc4{0, 0, 0, 0};
  if (tid == 0) {
    d.stats[0] = 0;
    d.stats[1] = 0;
    d.qctl[0] = 0;
    d.qctl[1] = 0;
  }
  const float4* phi = d.phi[phi_buf];
  for (int i = tid; i < d.V; i += stride) {
    float sg[4];
    const DQ H = blend_bones(sHd, d.bidx[i], d.bw[i], sg);
    const float4 x0 = d.v0[i], p = phi[i];
    const float3 v = dq_point(H, make_float3(x0.x + p.x, x0.y + p.y, x0.z + p.z));
    d.v[i] = make_float4(v.x, v.y, v.z, 0.f);
  }
}

// ctl (batches only): the first block resets the association's tile and tail counters of this iteration.
__global__ void __launch_bounds__(kBlock) k_skin(BatchGrid g, Dev d0, int phi_buf, unsigned* ctl) {
  if (g.map == nullptr) {
    skin_impl(d0, grid_pos(), phi_buf);
    return;
  }
  __shared__ Dev sd;
  if (ctl && blockIdx.x == 0 && threadIdx.x < 2) ctl[1 + threadIdx.x] = 0;  // tile and tail counters
  skin_impl(sd, batch_block(g, sd), phi_buf);
}

static int grid_for(int n, int block) { return (n + block - 1) / block; }

void launch_skin(const Dev& d, int phi_buf, cudaStream_t st) {
  const int g = max(grid_for(d.V, kBlock), 152);
  k_skin<<<g, kBlock, d.L * sizeof(DQ), st>>>(kSingle, d, phi_buf, nullptr);
}

// ---------------------------------------------------------------------------------------------
// z-buffer: one thread per triangle, pixel centres at integer coordinates, inclusive edge test for
// both windings, depth from the ray-plane intersection, min-reduced as (float bits << 32) | id.
// Also writes the unnormalised face normal (b - a) x (c - a) used by the vertex normals.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void raster_impl(const Dev& d, BlockPos bp) {
  const int f = bp.x * blockDim.x + threadIdx.x;
  if (f >= d.F) return;
  const int4 t = d.tris[f];
  const Cam c = d.cam;
  const float3 o = make_float3(c.ox, c.oy, c.oz);
  const float3 Al = f3(d.v[t.x]), Bl = f3(d.v[t.y]), Cl = f3(d.v[t.z]);
  const float3 N = cross3(sub3(Bl, Al), sub3(Cl, Al));
  d.fn[f] = make_float4(N.x, N.y, N.z, 0.f);
  const float3 A = make_float3(Al.x + o.x, Al.y + o.y, Al.z + o.z);  // camera frame
  const float3 B = make_float3(Bl.x + o.x, Bl.y + o.y, Bl.z + o.z);
  const float3 C = make_float3(Cl.x + o.x, Cl.y + o.y, Cl.z + o.z);
  if (A.z <= c.z_near || B.z <= c.z_near || C.z <= c.z_near) return;
  const float ua = c.fx * A.x / A.z + c.cx, va = c.fy * A.y / A.z + c.cy;
  const float ub = c.fx * B.x / B.z + c.cx, vb = c.fy * B.y / B.z + c.cy;
  const float uc = c.fx * C.x / C.z + c.cx, vc = c.fy * C.y / C.z + c.cy;
  if (!(isfinite(ua) && isfinite(ub) && isfinite(uc) && isfinite(va) && isfinite(vb) && isfinite(vc))) return;
  const float area = (ub - ua) * (vc - va) - (vb - va) * (uc - ua);
  if (area == 0.f) return;
  const float NA = dot3(N, A);
  const int x0 = (int)fmaxf(0.f, ceilf(fminf(ua, fminf(ub, uc))));
  const int x1 = (int)fminf((float)(c.W - 1), floorf(fmaxf(ua, fmaxf(ub, uc))));
  const int y0 = (int)fmaxf(0.f, ceilf(fminf(va, fminf(vb, vc))));
  const int y1 = (int)fminf((float)(c.H - 1), floorf(fmaxf(va, fmaxf(vb, vc))));
  for (int py = y0; py <= y1; ++py) {
    const float fy = (float)py;
    for (int px = x0; px <= x1; ++px) {
      const float fx = (float)px;
      const float w0 = (uc - ub) * (fy - vb) - (vc - vb) * (fx - ub);
      const float w1 = (ua - uc) * (fy - vc) - (va - vc) * (fx - uc);
      const float w2 = (ub - ua) * (fy - va) - (vb - va) * (fx - ua);
      const bool inside = (w0 >= 0.f && w1 >= 0.f && w2 >= 0.f) || (w0 <= 0.f && w1 <= 0.f && w2 <= 0.f);
      if (!inside) continue;
      const float dx = (fx - c.cx) / c.fx, dy = (fy - c.cy) / c.fy;
      const float den = N.x * dx + N.y * dy + N.z;
      if (den == 0.f) continue;
      const float z = NA / den;
      if (!(z > 0.f)) continue;
      const unsigned long long key = ((unsigned long long)__float_as_uint(z) << 32) | (unsigned)f;
      atomicMin(&d.zbuf[py * c.W + px], key);
    }
  }
}

__global__ void __launch_bounds__(kBlock) k_raster(BatchGrid g, Dev d0) {
  if (g.map == nullptr) {
    raster_impl(d0, grid_pos());
    return;
  }
  __shared__ Dev sd;
  raster_impl(sd, batch_block(g, sd));
}

// A batch's launch: registers sized for kBatchMinBlocks resident blocks (a few spills for occupancy).
__global__ void __launch_bounds__(kBlock, kBatchMinBlocks) k_raster_b(BatchGrid g) {
  __shared__ Dev sd;
  raster_impl(sd, batch_block(g, sd));
}

void launch_raster(const Dev& d, cudaStream_t st) {
  if (d.F > 0) k_raster<<<grid_for(d.F, kBlock), kBlock, 0, st>>>(kSingle, d);
}

// ---------------------------------------------------------------------------------------------
// Vertex normals (sum of incident face normals in face order, normalised), visibility (front-facing,
// rounded pixel inside the image, not behind the z-buffer by more than eps_vis), and insertion of
// each visible vertex into its pixel's bucket (a singly linked list: head[pixel] -> rec[i].w).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void visibility_impl(const Dev& d, BlockPos bp) {
  const int i = bp.x * blockDim.x + threadIdx.x;
  if (i >= d.V) return;
  float3 s = make_float3(0.f, 0.f, 0.f);
  const int b = d.csr_off[i], e = d.csr_off[i + 1];
  const float4 pl = d.v[i];
  // incident faces in groups of 8: all indices, then all normals in flight, then added in order
  for (int t0 = b; t0 < e; t0 += 8) {
    int f[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k] = t0 + k < e ? d.csr_face[t0 + k] : -1;
    float4 fn[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) fn[k] = f[k] >= 0 ? d.fn[f[k]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (f[k] >= 0) {
        s.x += fn[k].x;
        s.y += fn[k].y;
        s.z += fn[k].z;
      }
  }
  const float len = sqrtf(dot3(s, s));
  const bool valid = len >= 1e-12f;
  const float3 n = valid ? make_float3(s.x / len, s.y / len, s.z / len) : make_float3(0.f, 0.f, 0.f);
  d.n[i] = make_float4(n.x, n.y, n.z, valid ? 1.f : 0.f);
  int vp = -1;
  const Cam c = d.cam;
  const float3 p = make_float3(pl.x + c.ox, pl.y + c.oy, pl.z + c.oz);  // camera frame
  if (valid && p.z > c.z_near) {
    const float nd = dot3(n, p);
    const float u = c.fx * p.x / p.z + c.cx, vv = c.fy * p.y / p.z + c.cy;
    const float fu = floorf(u + 0.5f), fv = floorf(vv + 0.5f);
    if (nd < 0.f && fu >= 0.f && fv >= 0.f && fu < (float)c.W && fv < (float)c.H) {
      const int k = (int)fv * c.W + (int)fu;
      const unsigned long long key = d.zbuf[k];
      bool ok = true;
      if (key != ~0ull) ok = p.z <= __uint_as_float((unsigned)(key >> 32)) + c.eps_vis;
      if (ok) {
        vp = k;
        const int old = atomicExch(&d.head[k], i);
        d.rec[i] = make_float4(pl.x, pl.y, pl.z, __int_as_float(old));
        // the first vertex of a bucket is also stored with the pixel, so that a bucket holding one vertex
        // is read with two independent loads (head, pixrec) instead of a dependent chain
        if (old < 0) d.pixrec[k] = make_float4(pl.x, pl.y, pl.z, __int_as_float(i));
      }
    }
  }
  d.vispix[i] = vp;
}

__global__ void __launch_bounds__(kBlock) k_visibility(BatchGrid g, Dev d0) {
  if (g.map == nullptr) {
    visibility_impl(d0, grid_pos());
    return;
  }
  __shared__ Dev sd;
  visibility_impl(sd, batch_block(g, sd));
}

__global__ void __launch_bounds__(kBlock, kBatchMinBlocks) k_visibility_b(BatchGrid g) {
  __shared__ Dev sd;
  visibility_impl(sd, batch_block(g, sd));
}

void launch_visibility(const Dev& d, cudaStream_t st) {
  k_visibility<<<grid_for(d.V, kBlock), kBlock, 0, st>>>(kSingle, d);
}

// ---------------------------------------------------------------------------------------------
// Sec. 4.1 projective association.  Each valid pixel back-projects to p = ((px-cx) d/fx, (py-cy) d/fy, d)
// and takes the closest visible vertex (squared distance, ties to the smaller index) among the buckets
// of the (2W+1)^2 window, within the cutoff tau.  The window is searched in rings of growing Chebyshev
// radius r; after ring r every unvisited vertex lies at least d (r + 1/2) kappa away (it projects at
// least r + 1/2 pixels from the pixel, and kappa = min over axes of 1 / (f sqrt(1 + c_max^2)) turns
// that angle into a distance from p), so the search stops once that bound exceeds the best distance
// or tau: the result is the same argmin as the exhaustive window search.
//
// k_associate: rings 0..kRingsPerThread by the pixel's own thread, four buckets' heads and first records
// loaded together.  Pixels still open after that (the bound of ring 1 is ~4 mm at 2-3 m: pixels whose
// nearest vertex is farther, in the first iterations of a frame, at silhouettes and where vertices are
// sparse) go to a queue that the tail kernels drain with a group of lanes per pixel (a warp for one session,
// 4 lanes in a batch), the lanes splitting the next rings' buckets and combining (d^2, index) keys with a
// group min.
// The pixel's offset p - v_i is added to the vertex's fixed-point sums (integer atomics: the sums do
// not depend on the order of the additions).
// ---------------------------------------------------------------------------------------------
constexpr int kRingsPerThread = 1;

// The nearest candidate so far: its vertex (-1: none), squared distance and position (the record's, which
// holds the vertex's skinned position bit for bit, so the pixel's sums need no second load of it).
struct Best {
  int i;
  float d2;
  float3 v;
};

__device__ __forceinline__ void consider(int i, float3 p, float4 r, float tau2, Best& b) {
  const float dx = p.x - r.x, dy = p.y - r.y, dz = p.z - r.z;
  const float d2 = dx * dx + dy * dy + dz * dz;
  if (d2 <= tau2 && (b.i < 0 || d2 < b.d2 || (d2 == b.d2 && i < b.i))) {
    b.i = i;
    b.d2 = d2;
    b.v = make_float3(r.x, r.y, r.z);
  }
}

// bucket t (0 <= t < 8r) of the ring of Chebyshev radius r around (px, py), or -1 outside the image
__device__ __forceinline__ int ring_bucket(int px, int py, int r, int t, int W, int H) {
  int x, y;
  // top row: 2r+1 cells, bottom row: 2r+1, left column: 2r-1 (corners excluded), right column: 2r-1
  if (t <= 2 * r) { x = px - r + t; y = py - r; }
  else if (t <= 4 * r + 1) { x = px - r + (t - 2 * r - 1); y = py + r; }
  else if (t <= 6 * r) { x = px - r; y = py - r + 1 + (t - 4 * r - 2); }
  else { x = px + r; y = py - r + 1 + (t - 6 * r - 1); }
  return (x >= 0 && y >= 0 && x < W && y < H) ? y * W + x : -1;
}

// The rest of a bucket after its first record: walk from the head until the first record is reached.
__device__ __forceinline__ void scan_rest(const Dev& d, int h, int first, float3 p, float tau2, Best& best) {
  // a bucket list never holds more than |V| entries; the hop bound only guards against misuse
  for (int hops = 0; h >= 0 && h != first && hops < d.V; ++hops) {
    const float4 r = d.rec[h];
    consider(h, p, r, tau2, best);
    h = __float_as_int(r.w);
  }
}

// Scans up to N buckets whose pixel indices are in q[0..N) (-1 = none), every head and first record in
// flight at once.  The rest of the lists: one after the other (kSideBySide false: the fewest registers,
// for the thread-per-pixel pass whose occupancy pays more) or all N side by side, one load per list still
// open per round trip (a pixel then waits for its longest list, not for the sum of its lists).
template <int N, bool kSideBySide>
__device__ __forceinline__ void scan_group(const Dev& d, const int* q, float3 p, float tau2, Best& best) {
  int h[N], first[N];
  {
    float4 f[N];
#pragma unroll
    for (int u = 0; u < N; ++u) {
      h[u] = q[u] >= 0 ? __ldg(&d.head[q[u]]) : -1;
      f[u] = q[u] >= 0 ? d.pixrec[q[u]] : make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
    }
#pragma unroll
    for (int u = 0; u < N; ++u) {
      first[u] = __float_as_int(f[u].w);
      if (h[u] >= 0) consider(first[u], p, f[u], tau2, best);
      if (h[u] == first[u]) h[u] = -1;  // h[u]: the next record of list u still to visit (-1: none)
      if constexpr (!kSideBySide) {
        if (h[u] >= 0) scan_rest(d, h[u], first[u], p, tau2, best);
      }
    }
  }
  if constexpr (kSideBySide) {
    // a list never holds more than |V| entries; the round bound only guards against misuse
#pragma unroll 1
    for (int round = 0; round < d.V; ++round) {
      bool open = false;
#pragma unroll
      for (int u = 0; u < N; ++u) open |= h[u] >= 0;
      if (!open) break;
      float4 r[N];
#pragma unroll
      for (int u = 0; u < N; ++u)
        if (h[u] >= 0) r[u] = d.rec[h[u]];
#pragma unroll
      for (int u = 0; u < N; ++u)
        if (h[u] >= 0) {
          consider(h[u], p, r[u], tau2, best);
          const int next = __float_as_int(r[u].w);
          h[u] = (next == first[u] || next < 0) ? -1 : next;
        }
    }
  }
}

__device__ __forceinline__ unsigned long long key_of(int best, float bd2) {
  return best < 0 ? ~0ull : (((unsigned long long)__float_as_uint(bd2) << 32) | (unsigned)best);
}

// Adds pixel p's offset from its vertex (position vb) to the vertex's fixed-point sums.
__device__ __forceinline__ void commit_pixel(const Dev& d, int best, float3 p, float3 vb) {
  unsigned long long* a = reinterpret_cast<unsigned long long*>(&d.acc[best]);
  atomicAdd(a + 0, (unsigned long long)__float2ll_rn((p.x - vb.x) * kFix));
  atomicAdd(a + 1, (unsigned long long)__float2ll_rn((p.y - vb.y) * kFix));
  atomicAdd(a + 2, (unsigned long long)__float2ll_rn((p.z - vb.z) * kFix));
  atomicAdd(a + 3, 1ull);
}

__device__ __forceinline__ float3 back_project(const Cam& c, int px, int py, float dep) {
  // in FP64, then moved into the session-local frame (exact up to one FP32 rounding)
  return make_float3((float)(((double)px - (double)c.cx) * (double)dep * c.inv_fx - (double)c.ox),
                     (float)(((double)py - (double)c.cy) * (double)dep * c.inv_fy - (double)c.oy),
                     (float)((double)dep - (double)c.oz));
}

// One lane's pixel (px, py) of a warp's unit (active false: the lane has none; it still takes part in
// the warp's votes).
__device__ __forceinline__ void associate_impl(const Dev& d, int px, int py, bool active) {
  const Cam c = d.cam;
  const int lane = threadIdx.x & 31;
  const bool inimg = active && px < c.W && py < c.H;
  const int k = py * c.W + px;
  const float dep = inimg ? d.depth[k] : 0.f;
  const float tau2 = c.tau * c.tau;
  Best best{-1, 0.f, make_float3(0.f, 0.f, 0.f)};
  float3 p = make_float3(0.f, 0.f, 0.f);
  bool open = false;
  if (dep > 0.f && d.association == 1) {
    // the nearest corner of the triangle the z-buffer holds at this pixel (O(1), no queue)
    p = back_project(c, px, py, dep);
    const unsigned long long key = d.zbuf[k];
    if (key != ~0ull) {
      const int4 t = d.tris[(int)(unsigned)(key & 0xffffffffu)];
      consider(t.x, p, d.v[t.x], tau2, best);
      consider(t.y, p, d.v[t.y], tau2, best);
      consider(t.z, p, d.v[t.z], tau2, best);
    }
  } else if (dep > 0.f) {
    p = back_project(c, px, py, dep);
    open = true;
    if (c.R == 0) {
      const int q0[1] = {k};
      scan_group<1, false>(d, q0, p, tau2, best);
      open = false;
    } else {
      // rings 0 and 1 (9 buckets) in two rounds of independent loads: the pixel's own bucket with the
      // first four of ring 1, then the other four; the ring-1 bound decides whether the search goes on
      int q[5];
      q[0] = k;
#pragma unroll
      for (int u = 0; u < 4; ++u) q[1 + u] = ring_bucket(px, py, 1, u, c.W, c.H);
      scan_group<5, false>(d, q, p, tau2, best);
#pragma unroll
      for (int u = 0; u < 4; ++u) q[u] = ring_bucket(px, py, 1, 4 + u, c.W, c.H);
      scan_group<4, false>(d, q, p, tau2, best);
      const float lb = dep * (1.0f + 0.499f) * c.kappa;
      if (lb > c.tau || (best.i >= 0 && lb * lb > best.d2) || c.R == 1) open = false;
    }
  }
  // queue the open pixels (one atomic per warp)
  const unsigned om = __ballot_sync(0xffffffffu, open);
  unsigned base = 0;
  if (lane == 0 && om) base = atomicAdd(&d.qctl[0], __popc(om));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (open) d.queue[base + __popc(om & ((1u << lane) - 1u))] = make_int4(k, best.i, __float_as_int(best.d2), 0);
  if (inimg && !open) d.corr[k] = best.i;
  const bool done = !open && best.i >= 0;
  if (done) commit_pixel(d, best.i, p, best.v);
  const unsigned m = __ballot_sync(0xffffffffu, done);
  if (lane == 0 && m) atomicAdd(&d.stats[0], __popc(m));
}


constexpr int kTailWarps = 8;
constexpr int kTailPerLane = 4;       // buckets a lane loads at once (one session: a warp per pixel)
constexpr int kBatchTailLanes = 8;    // a batch's tail: lanes per queued pixel ...
constexpr int kBatchTailPerLane = 4;  // ... and buckets each of them loads at once

// The rings beyond the thread-owned ones for queue entry `item` of session d, by a group of GL lanes (lanes
// gl = lane % GL of the group starting at lane gbase, gmask naming them): the lanes split each
// ring's 8r buckets (up to kTailPerLane each per round trip, heads and first records loaded together) and
// combine (d^2, index) keys with a group min.  Returns, in every lane of the group, whether the pixel got a
// correspondence (its first lane writes it and adds the pixel's sums).
// One session's tail takes a warp per pixel (its queue is short and its latency is the slowest pixel's
// rings); a batch's takes 8 lanes per pixel (four pixels per warp: throughput over many queues).
template <int GL, int PL>
__device__ __forceinline__ bool tail_item(const Dev& d, unsigned item, int gl, unsigned gmask) {
  const Cam c = d.cam;
  const float tau2 = c.tau * c.tau;
  const int4 e = d.queue[item];
  const int k = e.x, px = k % c.W, py = k / c.W;
  const float dep = d.depth[k];
  const float3 p = back_project(c, px, py, dep);
  unsigned long long key = key_of(e.y, __int_as_float(e.z));
  Best w{-1, 0.f, make_float3(0.f, 0.f, 0.f)};
  // rings r0..r1 at a time, as many whole rings as the group's load slots hold (at least one): scanning
  // rings past the one whose bound ends the search only confirms the argmin, so the result is the same
  constexpr int kSlots = GL * PL;
  for (int r0 = kRingsPerThread + 1; r0 <= c.R;) {
    int r1 = r0, nb = 8 * r0;
    while (r1 < c.R && nb + 8 * (r1 + 1) <= kSlots) nb += 8 * ++r1;
    for (int t0 = 0; t0 < nb; t0 += kSlots) {
      int q[PL];
#pragma unroll
      for (int u = 0; u < PL; ++u) {
        int t = t0 + gl + GL * u, r = r0;
        while (t < nb && t >= 8 * r) t -= 8 * r++;  // bucket t of the group: ring r, position t
        q[u] = t0 + gl + GL * u < nb ? ring_bucket(px, py, r, t, c.W, c.H) : -1;
      }
      scan_group<PL, true>(d, q, p, tau2, w);
    }
    unsigned long long kk = key_of(w.i, w.d2);
    kk = kk < key ? kk : key;
#pragma unroll
    for (int o = GL / 2; o > 0; o >>= 1) {
      const unsigned long long other = __shfl_xor_sync(gmask, kk, o);
      kk = other < kk ? other : kk;
    }
    key = kk;
    const float lb = dep * ((float)r1 + 0.499f) * c.kappa;
    if (lb > c.tau || (key != ~0ull && lb * lb > __uint_as_float((unsigned)(key >> 32)))) break;
    r0 = r1 + 1;
  }
  const int best = key == ~0ull ? -1 : (int)(unsigned)(key & 0xffffffffu);
  if (gl == 0) {
    d.corr[k] = best;
    if (best >= 0) {
      const float4 vb = d.v[best];
      commit_pixel(d, best, p, make_float3(vb.x, vb.y, vb.z));
    }
  }
  return best >= 0;
}

// Persistent warps take the frame's association units (up to 32 pixels of a tile with a valid depth; one
// session's from k_tiles, a batch's from the depth gather), warp w the units w, w + (warps in the grid),
// ...: no counter and no block barrier, so a warp whose pixels are cheap goes on to its next unit at once,
// and the interleaving spreads the units of costly sessions over all warps.  In a batch each warp keeps
// its own copy of its unit's session descriptor in shared memory (reloaded when the session changes).
// Pixels outside the units keep the "no correspondence" the frame's depth copy wrote.
__global__ void __launch_bounds__(kBlock, kAssocBlocksPerSM) k_associate(const Dev* devs, const AssocUnit* units,
                                                                          const unsigned* ctl, Dev d0) {
  __shared__ Dev sd[kBlock / 32];
  const bool single = devs == nullptr;
  const unsigned n = single ? d0.qctl[2] : ctl[0];
  const AssocUnit* list = single ? d0.units : units;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned nw = gridDim.x * (kBlock / 32);
  if (single) {
#pragma unroll 1
    for (unsigned u = blockIdx.x * (kBlock / 32) + w; u < n; u += nw) {
      const int4 h = *reinterpret_cast<const int4*>(&list[u]);  // (session, x0, y0, pixels)
      const int o = lane < h.w ? list[u].off[lane] : 0;
      associate_impl(d0, h.y + (o & 15), h.z + (o >> 4), lane < h.w);
    }
    return;
  }
  int cur = -1;
#pragma unroll 1
  for (unsigned u = blockIdx.x * (kBlock / 32) + w; u < n; u += nw) {
    const int4 h = *reinterpret_cast<const int4*>(&list[u]);
    const int o = lane < h.w ? list[u].off[lane] : 0;
    if (h.x != cur) {
      __syncwarp();  // every lane is done with the previous descriptor
      const int* src = reinterpret_cast<const int*>(devs + h.x);
      for (int q = lane; q < (int)(sizeof(Dev) / 4); q += 32) reinterpret_cast<int*>(&sd[w])[q] = src[q];
      __syncwarp();
      cur = h.x;
    }
    associate_impl(sd[w], h.y + (o & 15), h.z + (o >> 4), lane < h.w);
  }
}

// One session: the warps of all blocks take its queue entries, warp w the w-th, then the rest from the
// session's counter (no counter traffic when the queue is no longer than the grid's warps).
__global__ void __launch_bounds__(32 * kTailWarps) k_associate_tail(Dev d) {
  const int lane = threadIdx.x & 31, gl = lane, gbase = 0;
  const unsigned gmask = 0xffffffffu;
  const unsigned n = *(volatile unsigned*)&d.qctl[0];
  const unsigned warps = gridDim.x * kTailWarps;  // warp w takes entry w first, then the counter's
  int done = 0;
  for (unsigned item = blockIdx.x * kTailWarps + (threadIdx.x >> 5); item < n;) {
    done += tail_item<32, kTailPerLane>(d, item, gl, gmask);
    if (warps >= n) break;
    unsigned next = 0;
    if (gl == 0) next = warps + atomicAdd(&d.qctl[1], 1u);
    item = __shfl_sync(gmask, next, gbase);
  }
  if (gl == 0 && done) atomicAdd(&d.stats[0], done);
}

// A batch: prefix[s] = queued pixels of the sessions before s (one block; at most 1024 x 4 sessions).
__global__ void __launch_bounds__(1024) k_tail_prefix(const Dev* devs, int n_sessions, unsigned* prefix) {
  __shared__ unsigned part[1024];
  const int t = threadIdx.x;
  unsigned v[4], sum = 0;
  for (int u = 0; u < 4; ++u) {
    const int s = 4 * t + u;
    v[u] = s < n_sessions ? *(volatile unsigned*)&devs[s].qctl[0] : 0u;
    sum += v[u];
  }
  part[t] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {  // inclusive scan of the per-thread sums
    const unsigned x = t >= o ? part[t - o] : 0u;
    __syncthreads();
    part[t] += x;
    __syncthreads();
  }
  unsigned run = part[t] - sum;
  for (int u = 0; u < 4; ++u) {
    const int s = 4 * t + u;
    if (s < n_sessions) prefix[s] = run;
    run += v[u];
  }
  if (t == 1023) prefix[n_sessions] = part[t];
}

// A batch: the lane groups take entries of the concatenated queues of all sessions, group g the g-th, then
// the rest from one counter; an entry's session is found in the prefix and its descriptor read through
// the cache.
__global__ void __launch_bounds__(32 * kTailWarps) k_associate_tail_batch(const Dev* devs, int n_sessions,
                                                                          const unsigned* prefix, unsigned* ctl) {
  constexpr int GL = kBatchTailLanes;
  const int lane = threadIdx.x & 31, gl = lane % GL, gbase = lane - gl;
  const unsigned gmask = ((1u << GL) - 1u) << gbase;
  const unsigned total = prefix[n_sessions];
  const unsigned groups = gridDim.x * (blockDim.x / GL);  // group g takes entry g first, then the counter's
  for (unsigned item = (blockIdx.x * blockDim.x + threadIdx.x) / GL; item < total;) {
    int lo = 0, hi = n_sessions - 1;  // the last session whose prefix is <= item
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (prefix[mid] <= item) lo = mid; else hi = mid - 1;
    }
    const Dev& d = devs[lo];
    if (tail_item<GL, kBatchTailPerLane>(d, item - prefix[lo], gl, gmask) && gl == 0) atomicAdd(&d.stats[0], 1);
    if (groups >= total) break;
    unsigned next = 0;
    if (gl == 0) next = groups + atomicAdd(&ctl[2], 1u);
    item = __shfl_sync(gmask, next, gbase);
  }
}

void launch_associate(const Dev& d, cudaStream_t st) {
  const int nunits = ((d.cam.W + 15) / 16) * ((d.cam.H + 1) / 2);
  k_associate<<<min((nunits + kBlock / 32 - 1) / (kBlock / 32), kAssocBlocksPerSM * 152), kBlock, 0, st>>>(nullptr, nullptr,
                                                                                                   nullptr, d);
  k_associate_tail<<<2 * 152, 32 * kTailWarps, 0, st>>>(d);
}

// Appends this block's tile's association units to list: its pixels with a valid depth, in row-major
// order, 32 per unit (one counter update per tile).
__device__ __forceinline__ void list_units(bool valid, int session, int tx, int ty, AssocUnit* list, unsigned* count) {
  __shared__ int s_warp[kBlock / 32];
  __shared__ unsigned s_first;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned m = __ballot_sync(0xffffffffu, valid);
  if (lane == 0) s_warp[w] = __popc(m);
  __syncthreads();
  int before = 0, total = 0;
#pragma unroll
  for (int q = 0; q < kBlock / 32; ++q) {
    before += q < w ? s_warp[q] : 0;
    total += s_warp[q];
  }
  if (total == 0) return;
  const int nu = (total + 31) / 32;
  if (threadIdx.x == 0) s_first = atomicAdd(count, (unsigned)nu);
  __syncthreads();
  if (valid) {
    const int r = before + __popc(m & ((1u << lane) - 1u));
    list[s_first + r / 32].off[r % 32] = (unsigned char)threadIdx.x;
  }
  if ((int)threadIdx.x < nu)
    *reinterpret_cast<int4*>(&list[s_first + threadIdx.x]) =
        make_int4(session, tx * 16, ty * 16, min(32, total - 32 * (int)threadIdx.x));
}

// One 16 x 16 tile per block: copies the frame's depth into the session's buffer, marks every pixel
// "no correspondence" (the association rewrites the pixels of its units each iteration) and lists the
// tile's units that hold a valid pixel.
__global__ void __launch_bounds__(kBlock) k_tiles(Dev d, const float* __restrict__ src) {
  const int gx = (d.cam.W + 15) / 16;
  const int tx = blockIdx.x % gx, ty = blockIdx.x / gx;
  const int px = tx * 16 + (threadIdx.x & 15), py = ty * 16 + (threadIdx.x >> 4);
  bool valid = false;
  if (px < d.cam.W && py < d.cam.H) {
    const int k = py * d.cam.W + px;
    const float z = src[k];
    const_cast<float*>(d.depth)[k] = z;
    d.corr[k] = -1;
    valid = z > 0.f;
  }
  list_units(valid, 0, tx, ty, d.units, &d.qctl[2]);
}

void launch_tiles(const Dev& d, const float* src, cudaStream_t st) {
  cudaMemsetAsync(d.qctl + 2, 0, sizeof(unsigned), st);
  k_tiles<<<((d.cam.W + 15) / 16) * ((d.cam.H + 15) / 16), kBlock, 0, st>>>(d, src);
}

// ---- batched launches (one launch over the blocks of all sessions of a batch) ---------------------
void launch_skin_b(const BatchGrid& g, int nblk, int max_links, int phi_buf, unsigned* ctl, cudaStream_t st) {
  if (nblk > 0) k_skin<<<nblk, kBlock, max_links * sizeof(DQ), st>>>(g, Dev{}, phi_buf, ctl);
}
void launch_raster_b(const BatchGrid& g, int nblk, cudaStream_t st) {
  if (nblk > 0) k_raster_b<<<nblk, kBlock, 0, st>>>(g);
}
void launch_visibility_b(const BatchGrid& g, int nblk, cudaStream_t st) {
  if (nblk > 0) k_visibility_b<<<nblk, kBlock, 0, st>>>(g);
}
void launch_associate_b(const Dev* devs, int n_sessions, const AssocUnit* tiles, unsigned* ctl, unsigned* prefix,
                        int assoc_blocks, int tail_blocks, cudaStream_t st) {
  k_associate<<<assoc_blocks, kBlock, 0, st>>>(devs, tiles, ctl, Dev{});
  k_tail_prefix<<<1, 1024, 0, st>>>(devs, n_sessions, prefix);
  k_associate_tail_batch<<<tail_blocks, 32 * kTailWarps, 0, st>>>(devs, n_sessions, prefix, ctl);
}

// Copies each session's depth frame from srcs[session] into the session's own depth buffer, one 16 x 16
// tile per block, marks every pixel "no correspondence" and lists the association units (16 x 2 pixels)
// that hold a valid depth.
__global__ void __launch_bounds__(kBlock) k_gather_depth_b(BatchGrid g, const float* const* srcs, AssocUnit* units,
                                                           unsigned* ctl) {
  const int4 m = g.map[blockIdx.x];
  const Dev& d = g.devs[m.x];
  const int px = m.y * 16 + (threadIdx.x & 15), py = m.z * 16 + (threadIdx.x >> 4);
  bool valid = false;
  if (px < d.cam.W && py < d.cam.H) {
    const int k = py * d.cam.W + px;
    const float z = srcs[m.x][k];
    const_cast<float*>(d.depth)[k] = z;
    d.corr[k] = -1;
    valid = z > 0.f;
  }
  list_units(valid, m.x, m.y, m.z, units, &ctl[0]);
}
void launch_gather_depth_b(const BatchGrid& g, int nblk, const float* const* srcs, AssocUnit* tiles, unsigned* ctl,
                           cudaStream_t st) {
  if (nblk > 0) k_gather_depth_b<<<nblk, kBlock, 0, st>>>(g, srcs, tiles, ctl);
}

__global__ void k_depth_from_zbuf(Dev d, float* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.cam.W * d.cam.H) return;
  const unsigned long long key = d.zbuf[k];
  out[k] = key == ~0ull ? 0.f : __uint_as_float((unsigned)(key >> 32));
}

void launch_depth_from_zbuf(const Dev& d, float* out, cudaStream_t st) {
  k_depth_from_zbuf<<<grid_for(d.cam.W * d.cam.H, kBlock), kBlock, 0, st>>>(d, out);
}

}  // namespace trk
